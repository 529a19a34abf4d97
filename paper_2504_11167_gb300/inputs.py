"""Seeded synthetic inputs for the LR-SPIKE workloads.

This module holds no part of the solver's arithmetic: it only draws the banded
matrices and right-hand sides that both the CUDA library's tests/benchmarks and
the CPU oracle consume.  Every generator uses numpy's PCG64 (``default_rng``)
with an explicit seed, so the same call gives the same bits on x86 and Arm.

Band storage everywhere is diagonal-major with 2k+1 rows:
``ab[k + i - j, j] = A[i, j]`` for ``|i - j| <= k`` (the LAPACK / scipy
``solve_banded`` convention with equal lower and upper bandwidth).
"""
from __future__ import annotations

import numpy as np

#: the seed of workload c is SEED_BASE + c
SEED_BASE = 111670


def _zero_outside(ab: np.ndarray, k: int) -> None:
    n = ab.shape[1]
    for d in range(2 * k + 1):
        off = d - k                       # row i = j + off
        if off > 0:
            ab[d, max(0, n - off):] = 0.0
        elif off < 0:
            ab[d, :min(n, -off)] = 0.0


def off_diagonal_row_sums(ab: np.ndarray, k: int) -> np.ndarray:
    """sum_{j != i} |A[i, j]| for every row i (entries outside the matrix are zero)."""
    n = ab.shape[1]
    s = np.zeros(n)
    for d in range(2 * k + 1):
        if d == k:
            continue
        off = d - k                       # A[j + off, j] = ab[d, j]
        lo, hi = max(0, -off), min(n, n - off)
        if hi > lo:
            s[lo + off:hi + off] += np.abs(ab[d, lo:hi])
    return s


def dominant_band(n: int, k: int, dom: float, seed: int) -> np.ndarray:
    """Random banded matrix: off-diagonal band entries uniform[-1, 1], and each
    diagonal entry dom * (sum of |off-diagonals| of its row), counting only
    entries inside the matrix.  dom > 1 gives strict diagonal dominance."""
    rng = np.random.default_rng(seed)
    ab = rng.uniform(-1.0, 1.0, size=(2 * k + 1, n))
    _zero_outside(ab, k)
    ab[k, :] = 0.0
    ab[k, :] = dom * off_diagonal_row_sums(ab, k)
    return ab


def dominant_band_torch(n: int, k: int, dom: float, seed: int, device="cuda"):
    """The recipe of dominant_band drawn with torch's generator on `device`
    (for workloads whose bands are too large to build on the host): entries
    uniform[-1, 1] inside the matrix, 0 outside, diagonal dom * (sum of
    |off-diagonals| of its row).  Not the same numbers as dominant_band."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    ab = torch.rand(2 * k + 1, n, generator=g, dtype=torch.float64, device=device) * 2.0 - 1.0
    j = torch.arange(n, device=device)
    rows = torch.zeros(n, dtype=torch.float64, device=device)
    for d in range(2 * k + 1):
        i = j + d - k                        # A[i, j] = ab[d, j]
        inside = (i >= 0) & (i < n)
        ab[d] = torch.where(inside, ab[d], torch.zeros_like(ab[d]))
        if d != k:
            lo, hi = max(0, k - d), min(n, n + k - d)
            rows[lo + d - k:hi + d - k] += ab[d, lo:hi].abs()
    ab[k] = dom * rows
    return ab


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides uniform[-1, 1], drawn from stream seed + 1; returned
    column-major (n x nrhs, Fortran order) so column q starts at q * n."""
    rng = np.random.default_rng(seed + 1)
    return rng.uniform(-1.0, 1.0, size=(nrhs, n)).T


def target(n: int, nrhs: int, seed: int) -> np.ndarray:
    """A seeded target vector x* uniform[-1, 1] from stream seed + 2 (for losses)."""
    rng = np.random.default_rng(seed + 2)
    return rng.uniform(-1.0, 1.0, size=(nrhs, n)).T


def low_rank_coupling_band(n: int, k: int, p: int, rank: int, dom: float, seed: int,
                           offsets: np.ndarray) -> np.ndarray:
    """A dominant band whose coupling blocks B_i and C_i all have rank <= ``rank``:
    the off-diagonal band entries that fall inside B_i (the last k rows of
    partition i, first k columns of partition i+1) and inside C_i are replaced
    by products of seeded random factors, kept triangular as the band forces,
    by making only the first ``rank`` rows (of B) / last ``rank`` columns (of C)
    nonzero."""
    ab = dominant_band(n, k, dom, seed)
    rng = np.random.default_rng(seed + 7)
    for i in range(p - 1):
        s = int(offsets[i + 1])
        # B_i[a, b] = A[s-k+a, s+b], nonzero only for b <= a; keep rows a >= k-rank
        for a in range(k):
            for b in range(a + 1):
                ab[k + (s - k + a) - (s + b), s + b] = rng.uniform(-1, 1) if a >= k - rank else 0.0
        # C_{i+1}[a, b] = A[s+a, s-k+b], nonzero only for a <= b; keep columns b < rank
        for a in range(k):
            for b in range(a, k):
                ab[k + (s + a) - (s - k + b), s - k + b] = rng.uniform(-1, 1) if b < rank else 0.0
    ab[k, :] = 0.0
    ab[k, :] = dom * off_diagonal_row_sums(ab, k)
    return ab


def convection_diffusion_band(nx: int, peclet: float) -> np.ndarray:
    """2-D convection-diffusion, 5-point stencil on an nx x nx interior grid,
    lexicographic order i = y*nx + x, scaled by h^2: diagonal 4, west and south
    neighbours -(1 + Pe), east and north -(1 - Pe), Dirichlet zero boundaries
    (boundary rows simply miss their outside neighbours).  Half-bandwidth nx."""
    n, k = nx * nx, nx
    ab = np.zeros((2 * k + 1, n))
    i = np.arange(n)
    x, y = i % nx, i // nx
    ab[k, :] = 4.0
    # A[i, i-1] (west) sits at ab[k + 1, i - 1]
    w = i[x > 0]
    ab[k + 1, w - 1] = -(1.0 + peclet)
    e = i[x < nx - 1]
    ab[k - 1, e + 1] = -(1.0 - peclet)
    s = i[y > 0]
    ab[2 * k, s - nx] = -(1.0 + peclet)
    nn = i[y < nx - 1]
    ab[0, nn + nx] = -(1.0 - peclet)
    return ab
