"""Plain FP64 CPU oracle of the LR-SPIKE hot path, written from the paper
(Spring, Polizzi, Sameh, "Low-Rank SPIKE Framework for Solving Large Sparse
Linear Systems with Applications", arXiv 2504.11167).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may use this module.  It shares no code with
the CUDA library; inputs come from ``paper_2504_11167_gb300.inputs``.

What it computes, step by step in the paper's order:
  * partitioning of the banded A into p diagonal blocks A_i with coupling
    blocks B_i, C_i (section 2.1, block-tridiagonal partition and the form of
    the off-diagonal blocks);
  * banded LU of every A_i (section 2.1 / 3.3, the D-stage factorisation), the
    plain C loops of ``band_ref.c``;
  * the right spike T_i = A_i^{-1}[0; B_i], i = 1..p-1, and the left spike
    W_i = A_i^{-1}[C_i; 0], i = 2..p (section 2.1, eq. 'Veqn');
  * rank-n_svd compression (section 3.1, eq. 'DiBaC' and the partitioned
    low-rank SVD that follows it): T_i ~ u Sigma v, W_i likewise.  Mode SPIKE
    takes the truncated SVD of the explicit spike; mode COUPLING takes the
    truncated SVD of B_i (C_i) and solves with its left factor, the
    alternative the paper discusses at the end of section 3.1.  For wide bands
    (k > 64) the truncation is the randomized SVD the paper uses (section 3.1,
    Halko-Martinsson-Tropp proto-algorithm with a few passes and oversampling),
    applied to the explicit spike: sketch, Householder QR, power passes,
    small SVD of Q^T T;
  * the reduced system of the low-rank spike matrix S~ = I + U V
    (section 3.2, eqs. 'per-partition_1/2' and 'red_sys_prec_mid_1'), in
    compressed unknowns zeta_i = P_i x_{i+1,t}, omega_{i+1} = Q_{i+1} x_{i,b}
    (the n_svd-sized exchanged vectors of section 3.2), assembled as the dense
    matrix R = I + V U and solved by dense LU.  FULL keeps all of R (the
    reduced system of LR-SPIKE-I, solved directly); TRUNCATED keeps only its
    per-interface diagonal blocks (S~~_r of eq. 'red_sys_prec_mid_2', the
    LR-SPIKE-T variant of section 3.3);
  * application of the preconditioner: D-stage g = D^{-1} f, reduced solve,
    recovery x_i = g_i - T~_i x_{i+1,t} - W~_i x_{i-1,b} (section 2.1, eqs.
    'D-stage-in-summary' .. 'recovery-stage-in-summary'; section 3.3 table
    'solver-list', low-rank recovery);
  * its transpose M^{-T} = D^{-T}(I - V^T R^{-T} U^T), derived from the same
    factorisation (the paper has no transposed solve);
  * the outer iteration: iterative refinement (the reduced-precision solver as
    a preconditioner of an iterative scheme, section 1) or right-preconditioned
    BiCGStab (section 3.3, table 'solver-list' caption).

Readings of places where the paper is silent or garbled are listed in the
repository's design notes; the ones that shape code here are commented inline.
"""
from __future__ import annotations

import ctypes
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg

from . import _cbuild

_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_i32 = _P(ctypes.c_int32)
_lib = None


def _c():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_cbuild.build())
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_band_lu_nopiv.argtypes = [i64, i32, _d, i64]
        lib.oracle_band_lu_nopiv.restype = ctypes.c_int
        lib.oracle_band_lu_piv.argtypes = [i64, i32, _d, i64, _i32]
        lib.oracle_band_lu_piv.restype = ctypes.c_int
        lib.oracle_band_solve_nopiv.argtypes = [i64, i32, _d, i64, _d, i64, i32, i32]
        lib.oracle_band_solve_piv.argtypes = [i64, i32, _d, i64, _i32, _d, i64, i32, i32]
        lib.oracle_band_matvec.argtypes = [i64, i32, _d, i64, _d, i64, _d, i64, i32, i32]
        _lib = lib
    return _lib


def _ptr(a, t=_d):
    return a.ctypes.data_as(t)


class SingularPivot(RuntimeError):
    """A zero or non-finite pivot met during a band LU."""


# --------------------------------------------------------------------------
# Band storage helpers.  ab has 2k+1 rows and n columns, ab[k + i - j, j] = A[i, j].
# --------------------------------------------------------------------------
def band_entry(ab: np.ndarray, k: int, i: int, j: int) -> float:
    if abs(i - j) > k:
        return 0.0
    return float(ab[k + i - j, j])


def band_to_dense(ab: np.ndarray, k: int) -> np.ndarray:
    n = ab.shape[1]
    A = np.zeros((n, n))
    for d in range(2 * k + 1):
        for j in range(n):
            i = j + d - k
            if 0 <= i < n:
                A[i, j] = ab[d, j]
    return A


def band_matvec(ab: np.ndarray, k: int, x: np.ndarray, trans: bool = False) -> np.ndarray:
    """Y = A X (or A^T X) for X of shape (n,) or (n, nrhs)."""
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    n = ab.shape[1]
    X = np.asfortranarray(np.atleast_2d(x.T).T, dtype=np.float64)
    Y = np.zeros_like(X, order="F")
    _c().oracle_band_matvec(n, k, _ptr(ab), n, _ptr(X), n, _ptr(Y), n, X.shape[1], int(trans))
    return Y.reshape(x.shape)


class BandLU:
    """LU factors of one banded block (plain loops in band_ref.c)."""

    def __init__(self, ab_block: np.ndarray, k: int, pivoting: bool):
        self.k, self.n, self.pivoting = k, ab_block.shape[1], pivoting
        if pivoting:
            store = np.zeros((3 * k + 1, self.n))
            store[k:, :] = ab_block
            self.ipiv = np.zeros(self.n, dtype=np.int32)
            info = _c().oracle_band_lu_piv(self.n, k, _ptr(store), self.n, _ptr(self.ipiv, _i32))
        else:
            store = np.array(ab_block, dtype=np.float64, order="C", copy=True)
            self.ipiv = None
            info = _c().oracle_band_lu_nopiv(self.n, k, _ptr(store), self.n)
        if info:
            raise SingularPivot(f"zero or non-finite pivot in column {info - 1}")
        self.store = store

    def solve(self, b: np.ndarray, trans: bool = False) -> np.ndarray:
        X = np.array(np.atleast_2d(b.T).T, dtype=np.float64, order="F", copy=True)
        if self.pivoting:
            _c().oracle_band_solve_piv(self.n, self.k, _ptr(self.store), self.n,
                                       _ptr(self.ipiv, _i32), _ptr(X), self.n, X.shape[1],
                                       int(trans))
        else:
            _c().oracle_band_solve_nopiv(self.n, self.k, _ptr(self.store), self.n, _ptr(X),
                                         self.n, X.shape[1], int(trans))
        return X.reshape(b.shape)


# --------------------------------------------------------------------------
# Partitioning (section 2.1): p blocks of roughly equal size, n_i > k.
# Reading: when p does not divide n, the first (n mod p) partitions get one
# extra row (the paper only asks for "roughly the same size").
# --------------------------------------------------------------------------
def partition_offsets(n: int, p: int) -> np.ndarray:
    base, extra = divmod(n, p)
    offs = [0]
    for i in range(p):
        offs.append(offs[-1] + base + (1 if i < extra else 0))
    return np.array(offs, dtype=np.int64)


def partition_band(ab: np.ndarray, k: int, s: int, m: int) -> np.ndarray:
    """Band of A_i = A[s:s+m, s:s+m]; entries that couple outside the block are dropped."""
    sub = np.array(ab[:, s:s + m], dtype=np.float64, copy=True)
    j = np.arange(m)
    for d in range(2 * k + 1):
        i = j + d - k
        sub[d, (i < 0) | (i >= m)] = 0.0
    return sub


def coupling_B(ab: np.ndarray, k: int, s_next: int) -> np.ndarray:
    """B_i: the k x k block of A in the last k rows of partition i and the first
    k columns of partition i+1 (section 2.1, form of the off-diagonal blocks)."""
    return np.array([[band_entry(ab, k, s_next - k + a, s_next + b) for b in range(k)]
                     for a in range(k)])


def coupling_C(ab: np.ndarray, k: int, s: int) -> np.ndarray:
    """C_i: the k x k block of A in the first k rows of partition i and the last
    k columns of partition i-1."""
    return np.array([[band_entry(ab, k, s + a, s - k + b) for b in range(k)] for a in range(k)])


# --------------------------------------------------------------------------
# Randomized truncation for wide bands (section 3.1: the randomized SVD of
# Halko, Martinsson and Tropp, "proto-algorithm", few passes, oversampling)
# --------------------------------------------------------------------------
_GOLDEN = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, i: int) -> int:
    """Output i (0-based) of the SplitMix64 generator started at `seed`
    (Steele, Lea and Flood, 2014): state_i = seed + (i+1)*0x9E3779B97F4A7C15,
    then the mixing function of the published definition."""
    z = (seed + (i + 1) * _GOLDEN) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def gaussian_sketch(rows: int, cols: int, seed: int) -> np.ndarray:
    """Omega (rows x cols): entry (a, j) is the Box-Muller normal of the
    SplitMix64 outputs 2c and 2c+1, c = a*cols + j, with
    u1 = ((o_2c >> 11) + 0.5) 2^-53 in (0, 1), u2 = (o_2c+1 >> 11) 2^-53:
    omega = sqrt(-2 ln u1) cos(2 pi u2).  A counter-based generator, so the
    CUDA side draws the same numbers from the same definition."""
    om = np.empty((rows, cols))
    for a in range(rows):
        for j in range(cols):
            c = a * cols + j
            u1 = ((splitmix64(seed, 2 * c) >> 11) + 0.5) * 2.0 ** -53
            u2 = (splitmix64(seed, 2 * c + 1) >> 11) * 2.0 ** -53
            om[a, j] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return om


def randomized_truncation(X: np.ndarray, r: int, ell: int, q: int, seed: int, rank_tol: float):
    """Rank-r truncation of X (n_i x k) by the randomized SVD of section 3.1
    (Halko, Martinsson and Tropp's proto-algorithm: a Gaussian sketch of ell =
    r + oversampling columns and q power passes), applied to X itself:

      Y = X Omega (Omega: k x ell Gaussian sketch);   Q = qr(Y)
      q times:   Y = X (X^T Q);   Q = qr(Y)          (re-orthonormalised pass)
      B = Q^T X  (ell x k);   B = U_B diag(s) V^T    (SVD)
      U = Q U_B,  keep the r largest s.

    qr is the Householder QR of LAPACK (numpy), the SVD LAPACK's.  With ell = k
    and X of rank k, Q spans range(X), Q Q^T X = X and the result is the exact
    truncated SVD.  Returns (U, sig, Vt, all singular values of B) like
    truncated_svd, with its rank guard."""
    k = X.shape[1]
    Q = np.linalg.qr(X @ gaussian_sketch(k, ell, seed))[0]
    for _ in range(q):
        Q = np.linalg.qr(X @ (X.T @ Q))[0]
    Ub, sv, Vt = np.linalg.svd(Q.T @ X, full_matrices=False)
    U, sig, V = np.zeros((X.shape[0], r)), np.zeros(r), np.zeros((r, k))
    for j in range(min(r, sv.size)):
        if sv[0] > 0.0 and sv[j] > rank_tol * sv[0]:
            U[:, j], sig[j], V[j, :] = Q @ Ub[:, j], sv[j], Vt[j, :]
    return U, sig, V, sv


def sketch_seed(base: int, part: int, side: int) -> int:
    """Seed of the sketch of partition `part`'s right (side 0) or left
    (side 1) spike."""
    return (base + 2 * part + side) & _M64


SKETCH_SEED = 0x4C52535049
WIDE_K = 64   # bands with k > WIDE_K are truncated by the randomized SVD


def truncated_svd(X: np.ndarray, r: int, rank_tol: float):
    """Rank-r truncated SVD X ~ U diag(sig) Vt, the 'low-rank SVD' of section 3.1.

    Rank guard (the paper reduces n_svd when singular values are near zero,
    section 4.2, without a threshold): a singular value sigma_j <= rank_tol *
    sigma_1 is dropped, i.e. its column of U and row of Vt are set to zero.
    Returns U (m x r), sig (r), Vt (r x ncols) and the full singular values."""
    Uf, s, Vt = np.linalg.svd(X, full_matrices=False)
    m, nc = X.shape
    U, sig, V = np.zeros((m, r)), np.zeros(r), np.zeros((r, nc))
    for j in range(min(r, s.size)):
        if s[0] > 0.0 and s[j] > rank_tol * s[0]:
            U[:, j], sig[j], V[j, :] = Uf[:, j], s[j], Vt[j, :]
    return U, sig, V, s


# --------------------------------------------------------------------------
# LR-SPIKE factorisation
# --------------------------------------------------------------------------
@dataclass
class Factor:
    n: int
    k: int
    p: int
    r: int
    offs: np.ndarray
    compress: str
    reduced: str
    parts: List[BandLU]
    UV: List[Optional[np.ndarray]]      # n_i x r, the u-factor of T~_i (None for i = p)
    PV: List[Optional[np.ndarray]]      # r x k, Sigma v of T~_i
    UW: List[Optional[np.ndarray]]      # n_i x r, the u-factor of W~_i (None for i = 1)
    QW: List[Optional[np.ndarray]]      # r x k, Sigma v of W~_i
    sigV: List[Optional[np.ndarray]] = field(default_factory=list)
    sigW: List[Optional[np.ndarray]] = field(default_factory=list)
    R: Optional[np.ndarray] = None      # the reduced matrix that is solved (FULL or TRUNCATED)
    R_full: Optional[np.ndarray] = None
    R_lu: object = None
    threads: int = 1

    @property
    def nz(self) -> int:
        return 2 * self.r * (self.p - 1)


def factor(ab: np.ndarray, k: int, p: int, r: int, compress: str = "spike",
           reduced: str = "full", pivoting: bool = False, rank_tol: float = 1e-13,
           threads: int = 1, randomized: Optional[bool] = None, oversample: Optional[int] = None,
           power_iters: int = 2, seed: int = SKETCH_SEED) -> Factor:
    """LR-SPIKE factorisation of the banded A (FP64).

    compress: "spike" (truncated SVD of the explicit spikes, section 3.1) or
              "coupling" (truncated SVD of B_i / C_i, then solves, section 3.1's
              alternative).
    reduced:  "full" (R = I + V U solved directly) or "truncated" (its
              per-interface diagonal blocks only, LR-SPIKE-T).
    pivoting: partial pivoting inside each partition (rows never cross
              partitions); B_i and C_i are taken from the unpivoted A.
    randomized: truncate the explicit spikes with randomized_truncation
              (default: when k > WIDE_K), ell = min(k, r + oversample)
              (oversample defaults to r), power_iters passes, sketch seeds
              sketch_seed(seed, i, side).
    """
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    n = ab.shape[1]
    assert ab.shape[0] == 2 * k + 1
    if not (p >= 1 and 0 <= r <= k):
        raise ValueError("need p >= 1 and 0 <= r <= k")
    offs = partition_offsets(n, p)
    sizes = np.diff(offs)
    if p > 1 and sizes.min() <= k:
        raise ValueError("every partition needs n_i > k (section 2.1)")
    if compress not in ("spike", "coupling") or reduced not in ("full", "truncated"):
        raise ValueError("bad mode")

    if randomized is None:
        randomized = k > WIDE_K
    ell = min(k, r + (r if oversample is None else oversample))

    def trunc(X, i, side):
        if randomized and compress == "spike":
            return randomized_truncation(X, r, ell, power_iters, sketch_seed(seed, i, side), rank_tol)
        return truncated_svd(X, r, rank_tol)

    def one(i):
        s, m = int(offs[i]), int(sizes[i])
        lu = BandLU(partition_band(ab, k, s, m), k, pivoting)
        out = [lu, None, None, None, None, None, None]
        if i < p - 1:                           # right spike T_i, i = 1..p-1 (eq. 'Veqn')
            B = coupling_B(ab, k, s + m)
            rhs = np.zeros((m, k))
            if compress == "spike":
                rhs[m - k:, :] = B
                U, sig, Vt, sv = trunc(lu.solve(rhs), i, 0)
                out[1], out[2], out[5] = U, sig[:, None] * Vt, sv
            else:
                Ub, sig, Vt, sv = truncated_svd(B, r, rank_tol)
                rhs2 = np.zeros((m, r))
                rhs2[m - k:, :] = Ub
                out[1], out[2], out[5] = lu.solve(rhs2), sig[:, None] * Vt, sv
        if i > 0:                               # left spike W_i, i = 2..p
            C = coupling_C(ab, k, s)
            if compress == "spike":
                rhs = np.zeros((m, k))
                rhs[:k, :] = C
                U, sig, Vt, sv = trunc(lu.solve(rhs), i, 1)
                out[3], out[4], out[6] = U, sig[:, None] * Vt, sv
            else:
                Uc, sig, Vt, sv = truncated_svd(C, r, rank_tol)
                rhs2 = np.zeros((m, r))
                rhs2[:k, :] = Uc
                out[3], out[4], out[6] = lu.solve(rhs2), sig[:, None] * Vt, sv
        return out

    if threads > 1:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(one, range(p)))
    else:
        res = [one(i) for i in range(p)]
    fac = Factor(n=n, k=k, p=p, r=r, offs=offs, compress=compress, reduced=reduced,
                 parts=[x[0] for x in res], UV=[x[1] for x in res], PV=[x[2] for x in res],
                 UW=[x[3] for x in res], QW=[x[4] for x in res],
                 sigV=[x[5] for x in res], sigW=[x[6] for x in res], threads=threads)
    if fac.nz:
        fac.R_full = assemble_R(fac)
        if reduced == "full":
            fac.R = fac.R_full
        else:
            fac.R = truncate_R(fac.R_full, r, p)
        fac.R_lu = scipy.linalg.lu_factor(fac.R)
    return fac


# --------------------------------------------------------------------------
# The compressed reduced system.  Reduced unknowns are ordered per interface
# i = 1..p-1 as z_i = [zeta_i ; omega_{i+1}] with zeta_i = P_i x_{i+1,t} and
# omega_{i+1} = Q_{i+1} x_{i,b} (section 3.2: the r-vectors v~ x that replace the
# k-row tips in the exchange).  "t" = first k rows, "b" = last k rows of a
# partition (section 2.1, tips).
# --------------------------------------------------------------------------
def V_op(fac: Factor, x: np.ndarray) -> np.ndarray:
    """z = V x: the projections of the tips that the low-rank spikes act on."""
    k, r, offs = fac.k, fac.r, fac.offs
    X = x.reshape(fac.n, -1)
    z = np.zeros((fac.nz, X.shape[1]))
    for i in range(fac.p - 1):
        s_next = int(offs[i + 1])
        z[2 * r * i: 2 * r * i + r] = fac.PV[i] @ X[s_next: s_next + k]          # P_i x_{i+1,t}
        z[2 * r * i + r: 2 * r * (i + 1)] = fac.QW[i + 1] @ X[s_next - k: s_next]  # Q_{i+1} x_{i,b}
    return z


def U_op(fac: Factor, z: np.ndarray) -> np.ndarray:
    """x = U z: x_i = u_{T,i} zeta_i + u_{W,i} omega_i (the low-rank spike columns)."""
    r, offs = fac.r, fac.offs
    Z = z.reshape(fac.nz, -1)
    x = np.zeros((fac.n, Z.shape[1]))
    for i in range(fac.p):
        s, e = int(offs[i]), int(offs[i + 1])
        if i < fac.p - 1:
            x[s:e] += fac.UV[i] @ Z[2 * r * i: 2 * r * i + r]
        if i > 0:
            x[s:e] += fac.UW[i] @ Z[2 * r * (i - 1) + r: 2 * r * i]
    return x


def V_op_T(fac: Factor, z: np.ndarray) -> np.ndarray:
    k, r, offs = fac.k, fac.r, fac.offs
    Z = z.reshape(fac.nz, -1)
    x = np.zeros((fac.n, Z.shape[1]))
    for i in range(fac.p - 1):
        s_next = int(offs[i + 1])
        x[s_next: s_next + k] += fac.PV[i].T @ Z[2 * r * i: 2 * r * i + r]
        x[s_next - k: s_next] += fac.QW[i + 1].T @ Z[2 * r * i + r: 2 * r * (i + 1)]
    return x


def U_op_T(fac: Factor, x: np.ndarray) -> np.ndarray:
    r, offs = fac.r, fac.offs
    X = x.reshape(fac.n, -1)
    z = np.zeros((fac.nz, X.shape[1]))
    for i in range(fac.p):
        s, e = int(offs[i]), int(offs[i + 1])
        if i < fac.p - 1:
            z[2 * r * i: 2 * r * i + r] += fac.UV[i].T @ X[s:e]
        if i > 0:
            z[2 * r * (i - 1) + r: 2 * r * i] += fac.UW[i].T @ X[s:e]
    return z


def assemble_R(fac: Factor, chunk: int = 256) -> np.ndarray:
    """R = I + V U, built column by column from the two operators."""
    nz = fac.nz
    R = np.eye(nz)
    for c0 in range(0, nz, chunk):
        c1 = min(nz, c0 + chunk)
        E = np.zeros((nz, c1 - c0))
        E[np.arange(c0, c1), np.arange(c1 - c0)] = 1.0
        R[:, c0:c1] += V_op(fac, U_op(fac, E))
    return R


def truncate_R(R: np.ndarray, r: int, p: int) -> np.ndarray:
    """Keep only the 2r x 2r diagonal blocks (one per interface), eq. 'red_sys_prec_mid_2'."""
    Rt = np.zeros_like(R)
    for i in range(p - 1):
        sl = slice(2 * r * i, 2 * r * (i + 1))
        Rt[sl, sl] = R[sl, sl]
    return Rt


# --------------------------------------------------------------------------
# Applying the preconditioner M^{-1} and its transpose
# --------------------------------------------------------------------------
def _per_partition(fac: Factor, fn):
    if fac.threads > 1:
        with ThreadPoolExecutor(fac.threads) as ex:
            return list(ex.map(fn, range(fac.p)))
    return [fn(i) for i in range(fac.p)]


def d_solve(fac: Factor, f: np.ndarray, trans: bool = False) -> np.ndarray:
    """D-stage: g_i = A_i^{-1} f_i (or A_i^{-T} f_i) for every partition."""
    F = f.reshape(fac.n, -1)
    offs = fac.offs
    parts = _per_partition(fac, lambda i: fac.parts[i].solve(F[offs[i]:offs[i + 1]], trans))
    return np.concatenate(parts, axis=0).reshape(f.shape)


def apply(fac: Factor, f: np.ndarray) -> np.ndarray:
    """x = M^{-1} f: D-stage, reduced solve, low-rank recovery (section 2.1 summary
    of the solve; section 3.3, LR-SPIKE-I / -T recovery with T~_i and W~_i)."""
    g = d_solve(fac, f)
    if fac.nz == 0:
        return g
    psi = V_op(fac, g)
    z = scipy.linalg.lu_solve(fac.R_lu, psi)
    return (g.reshape(fac.n, -1) - U_op(fac, z)).reshape(f.shape)


def apply_T(fac: Factor, h: np.ndarray) -> np.ndarray:
    """lambda = M^{-T} h = D^{-T}(h - V^T R^{-T} U^T h)."""
    if fac.nz == 0:
        return d_solve(fac, h, trans=True)
    a = U_op_T(fac, h)
    w = scipy.linalg.lu_solve(fac.R_lu, a, trans=1)
    y = h.reshape(fac.n, -1) - V_op_T(fac, w)
    return d_solve(fac, y, trans=True).reshape(h.shape)


# --------------------------------------------------------------------------
# Outer iterations (FP64).  Convergence is per right-hand side: every column
# must reach ||f - A x||_2 / ||f||_2 <= tol.
# --------------------------------------------------------------------------
@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    rel_residual: np.ndarray
    history: list
    converged: bool


def ir_solve(ab, k, fac: Factor, f: np.ndarray, tol: float = 1e-12, max_iter: int = 50,
             trans: bool = False) -> SolveResult:
    """Iterative refinement with M as the preconditioner: x += M^{-1}(f - A x)."""
    F = f.reshape(fac.n, -1)
    fn = np.linalg.norm(F, axis=0)
    fn[fn == 0] = 1.0
    x = np.zeros_like(F)
    hist = []
    prec = apply_T if trans else apply
    for it in range(max_iter + 1):
        res = F - band_matvec(ab, k, x, trans=trans)
        rel = np.linalg.norm(res, axis=0) / fn
        hist.append(rel.copy())
        if np.all(rel <= tol):
            return SolveResult(x.reshape(f.shape), it, rel, hist, True)
        if it == max_iter:
            break
        x = x + prec(fac, res)
    return SolveResult(x.reshape(f.shape), max_iter, rel, hist, False)


def bicgstab(ab, k, fac: Factor, f: np.ndarray, tol: float = 1e-12, max_iter: int = 200,
             trans: bool = False) -> SolveResult:
    """Right-preconditioned BiCGStab (van der Vorst), one column at a time.
    One iteration applies the preconditioner twice."""
    F = f.reshape(fac.n, -1)
    X = np.zeros_like(F)
    prec = apply_T if trans else apply
    rels, its, ok = [], 0, True
    for q in range(F.shape[1]):
        b = F[:, q]
        bn = np.linalg.norm(b) or 1.0
        x = np.zeros_like(b)
        r = b.copy()
        rh = r.copy()
        rho = alpha = omega = 1.0
        v = np.zeros_like(b)
        pv = np.zeros_like(b)
        rel = np.linalg.norm(r) / bn
        it = 0
        while rel > tol and it < max_iter:
            it += 1
            rho_new = rh @ r
            beta = (rho_new / rho) * (alpha / omega)
            pv = r + beta * (pv - omega * v)
            ph = prec(fac, pv)
            v = band_matvec(ab, k, ph, trans=trans)
            alpha = rho_new / (rh @ v)
            s = r - alpha * v
            if np.linalg.norm(s) / bn <= tol:
                x = x + alpha * ph
                r = s
                rel = np.linalg.norm(b - band_matvec(ab, k, x, trans=trans)) / bn
                break
            sh = prec(fac, s)
            t = band_matvec(ab, k, sh, trans=trans)
            omega = (t @ s) / (t @ t)
            x = x + alpha * ph + omega * sh
            r = s - omega * t
            rho = rho_new
            rel = np.linalg.norm(b - band_matvec(ab, k, x, trans=trans)) / bn
        X[:, q] = x
        rels.append(rel)
        its = max(its, it)
        ok = ok and rel <= tol
    return SolveResult(X.reshape(f.shape), its, np.array(rels), [], ok)


# --------------------------------------------------------------------------
# LR-SPIKE-OTF (section 2.2, "SPIKE-on-the-fly", eqs. 'OTF-1' and 'OTF-2';
# section 3.3: the truncated low-rank reduced system as its preconditioner).
# The TRUE reduced system of the spike matrix S = D^{-1} A is solved
# iteratively on the interface tips y_i = [x_{i,b} ; x_{i+1,t}] (2k per
# interface i = 1..p-1).  A product with the spikes is never formed: the spike
# terms of partition i act through one solve with A_i on the vector
#     c_i = [C_i x_{i-1,b} ; 0 ; B_i x_{i+1,t}]
# (eqs. OTF-1/OTF-2 applied right to left, both spikes at once by linearity):
#     (S_red y)_i = y_i + tips(A^{-1} c(y))_i.
# The preconditioner is S~~_r restricted to one interface,
#     [[I, T~_{i,b}], [W~_{i+1,t}, I]],  T~_{i,b} = u_{T,i}^(b) P_i, W~_{i+1,t} = u_{W,i+1}^(t) Q_{i+1},
# inverted by Woodbury through the 2r x 2r block E_i of the truncated reduced
# matrix.  Reduced BiCGStab to a tolerance (1e-8 by default, as in the paper's
# experiments), then the recovery x = g - A^{-1} c(y) with g = D^{-1} f.
# --------------------------------------------------------------------------
def otf_tips(fac: Factor, v: np.ndarray) -> np.ndarray:
    """Interface tips of a full vector: y_i = [v(s_{i+1}-k : s_{i+1}) ; v(s_{i+1} : s_{i+1}+k)]."""
    k, offs = fac.k, fac.offs
    V = v.reshape(fac.n, -1)
    y = np.zeros((fac.p - 1, 2 * k, V.shape[1]))
    for i in range(fac.p - 1):
        s = int(offs[i + 1])
        y[i, :k] = V[s - k: s]
        y[i, k:] = V[s: s + k]
    return y


def otf_coupling(fac: Factor, ab: np.ndarray, y: np.ndarray) -> np.ndarray:
    """c_i = [C_i x_{i-1,b} ; 0 ; B_i x_{i+1,t}] for all partitions (zero elsewhere)."""
    k, offs = fac.k, fac.offs
    c = np.zeros((fac.n, y.shape[2]))
    for i in range(fac.p - 1):
        s = int(offs[i + 1])
        B = coupling_B(ab, k, s)          # rows s-k..s-1, columns s..s+k-1
        C = coupling_C(ab, k, s)          # rows s..s+k-1, columns s-k..s-1
        c[s - k: s] += B @ y[i, k:]       # B_i x_{i+1,t} on the bottom rows of partition i
        c[s: s + k] += C @ y[i, :k]       # C_{i+1} x_{i,b} on the top rows of partition i+1
    return c


def otf_S(fac: Factor, ab: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The true reduced operator applied on the fly: y + tips(D^{-1} c(y))."""
    return y + otf_tips(fac, d_solve(fac, otf_coupling(fac, ab, y)))


def otf_prec(fac: Factor, y: np.ndarray) -> np.ndarray:
    """S~~_r^{-1} per interface (Woodbury): out = y - [u_T^(b) ; u_W^(t)] E_i^{-1} [P_i y_t ; Q_{i+1} y_b]."""
    k, r, offs = fac.k, fac.r, fac.offs
    out = y.copy()
    for i in range(fac.p - 1):
        s = int(offs[i + 1])
        si = int(offs[i])
        sl = slice(2 * r * i, 2 * r * (i + 1))
        E = fac.R_full[sl, sl]
        w = np.concatenate([fac.PV[i] @ y[i, k:], fac.QW[i + 1] @ y[i, :k]], axis=0)
        z = np.linalg.solve(E, w)
        out[i, :k] -= fac.UV[i][s - k - si: s - si] @ z[:r]          # u_T of partition i, bottom rows
        out[i, k:] -= fac.UW[i + 1][0:k] @ z[r:]                      # u_W of partition i+1, top rows
    return out


def otf_bicgstab(fac: Factor, ab: np.ndarray, b: np.ndarray, tol: float, max_iter: int):
    """Right-preconditioned BiCGStab on S_red y = b, column by column (the
    reduced residual |b - S_red y| / |b| <= tol).  Returns y and the largest
    iteration count."""
    Y = np.zeros_like(b)
    its = 0
    for q in range(b.shape[2]):
        bq = b[:, :, q:q + 1]
        bn = np.linalg.norm(bq) or 1.0
        y = np.zeros_like(bq)
        r = bq.copy()
        rh = r.copy()
        rho = alpha = omega = 1.0
        v = np.zeros_like(bq)
        pv = np.zeros_like(bq)
        it = 0
        while np.linalg.norm(r) / bn > tol and it < max_iter:
            it += 1
            rho_new = float(np.sum(rh * r))
            beta = (rho_new / rho) * (alpha / omega)
            pv = r + beta * (pv - omega * v)
            ph = otf_prec(fac, pv)
            v = otf_S(fac, ab, ph)
            alpha = rho_new / float(np.sum(rh * v))
            s = r - alpha * v
            sh = otf_prec(fac, s)
            t = otf_S(fac, ab, sh)
            tt = float(np.sum(t * t))
            omega = float(np.sum(t * s)) / tt if tt > 0 else 0.0
            y = y + alpha * ph + omega * sh
            r = s - omega * t
            rho = rho_new
        Y[:, :, q:q + 1] = y
        its = max(its, it)
    return Y, its


def otf_apply(fac: Factor, ab: np.ndarray, f: np.ndarray, otf_tol: float = 1e-8, max_iter: int = 100):
    """One LR-SPIKE-OTF solve: g = D^{-1} f; BiCGStab on S_red y = tips(g);
    x = g - D^{-1} c(y).  Returns x and the reduced iteration count."""
    g = d_solve(fac, f).reshape(fac.n, -1)
    if fac.p < 2:
        return g.reshape(f.shape), 0
    y, its = otf_bicgstab(fac, ab, otf_tips(fac, g), otf_tol, max_iter)
    x = g - d_solve(fac, otf_coupling(fac, ab, y))
    return x.reshape(f.shape), its


def otf_solve(ab, k, fac: Factor, f: np.ndarray, tol: float = 1e-12, max_iter: int = 20,
              otf_tol: float = 1e-8) -> SolveResult:
    """Outer refinement around OTF solves (the paper lowers the reduced tolerance
    and restarts when the solution is not accurate enough; here every extra
    pass solves for the correction of the current residual)."""
    F = f.reshape(fac.n, -1)
    fn = np.linalg.norm(F, axis=0)
    fn[fn == 0] = 1.0
    x = np.zeros_like(F)
    hist = []
    for it in range(max_iter + 1):
        res = F - band_matvec(ab, k, x)
        rel = np.linalg.norm(res, axis=0) / fn
        hist.append(rel.copy())
        if np.all(rel <= tol):
            return SolveResult(x.reshape(f.shape), it, rel, hist, True)
        if it == max_iter:
            break
        d, _ = otf_apply(fac, ab, res, otf_tol)
        x = x + d.reshape(x.shape)
    return SolveResult(x.reshape(f.shape), max_iter, rel, hist, False)


# --------------------------------------------------------------------------
# Gradient of a solve (the adjoint): x = A^{-1} f, L(x);  A^T lambda = dL/dx,
# dL/df = lambda, dL/dA = -lambda x^T (band entries only)
# --------------------------------------------------------------------------
def solve_gradients(ab: np.ndarray, k: int, f: np.ndarray, gx_of_x):
    """Exact x = A^{-1} f (LAPACK banded solve), lambda = A^{-T} gx_of_x(x),
    and the band gradient G[k + i - j, j] = -sum_q lambda[i, q] x[j, q]
    (zero outside the matrix).  f: (n,) or (n, nrhs)."""
    n = ab.shape[1]
    F = f.reshape(n, -1)
    x = scipy.linalg.solve_banded((k, k), ab, F)
    abT = np.zeros_like(ab)                 # band of A^T: A^T[i][j] = A[j][i]
    for d in range(2 * k + 1):
        off = d - k                         # A[j + off, j] = ab[d, j]  ->  A^T[j, j + off]
        for j in range(n):
            i = j + off
            if 0 <= i < n:
                abT[k + j - i, i] = ab[d, j]
    lam = scipy.linalg.solve_banded((k, k), abT, np.asarray(gx_of_x(x.reshape(f.shape))).reshape(n, -1))
    G = np.zeros_like(ab)
    for d in range(2 * k + 1):
        for j in range(n):
            i = j + d - k
            if 0 <= i < n:
                G[d, j] = -np.dot(lam[i, :], x[j, :])
    return x.reshape(f.shape), lam.reshape(f.shape), G

