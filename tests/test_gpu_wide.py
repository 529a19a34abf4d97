"""Wide bands (64 < k <= 1024) on the GPU: blocks of W = 64 ceil(k/64), block
products as batched GEMMs, randomized truncation of the spikes.

Parity: one FP64 preconditioner application against the oracle with the same
randomized truncation (same sketches: SplitMix64 + Box-Muller, seeds
0x4C52535049 + 2i + side, ell = 2r, two power passes, orthonormalisation cut
1e-7).  The two sides agree to rounding except where the Gram route's
resolution (~1e-4 sigma_1, see the oracle's pins) lets rounding differences
into the weakest kept directions, so the bound is 1e-9 instead of 1e-12.
Mixed FP32 and TF32 solves: relative residual <= 1e-10 per column (IR, or
BiCGStab where IR stalls), recomputed with the oracle's FP64 band product.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def gpu_solve(torch, ab, f, k, p, r, transpose=False, allow_unconverged=False, **kw):
    from paper_2504_11167_gb300.solver import LRSpike
    n = ab.shape[1]
    band = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(np.atleast_2d(f.T))).cuda()
    with LRSpike(n, k, p, r, **kw) as s:
        s.factor(band)
        x, info = (s.solve_transpose if transpose else s.solve)(ft, allow_unconverged=allow_unconverged)
        out = x.cpu().numpy().T.copy()
    return out.reshape(f.shape), info


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # n, k, p, r, dom, reduced, nrhs
    (6000, 96, 4, 8, 1.2, "truncated", 1),     # W = 128
    (5000, 70, 3, 6, 1.3, "full", 2),          # W = 128 > k, ragged partitions
    (20000, 200, 5, 16, 1.1, "truncated", 3),  # W = 256: two levels of recursive halving
    (3000, 100, 1, 4, 1.5, "full", 1),         # p = 1: the wide band LU alone
]


def case_id(c):
    return "n{}-k{}-p{}-r{}-{}-q{}".format(c[0], c[1], c[2], c[3], c[5], c[6])


@pytest.mark.parametrize("case", CASES, ids=[case_id(c) for c in CASES])
def test_wide_preconditioner_parity_fp64(torch_cuda, case):
    n, k, p, r, dom, reduced, nrhs = case
    seed = 2000 + n + k
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, nrhs, seed)
    fac = O.factor(ab, k, p, r, reduced=reduced)          # k > 64: randomized truncation
    got, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, outer="none")
    assert rel(got, O.apply(fac, np.asarray(f))) <= 1e-9
    gotT, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, outer="none", transpose=True)
    assert rel(gotT, O.apply_T(fac, np.asarray(f))) <= 1e-9


@pytest.mark.parametrize("precision", ["fp32", "tf32", "fp64"])
@pytest.mark.parametrize("transpose", [False, True])
def test_wide_solve_reaches_tolerance(torch_cuda, precision, transpose):
    n, k, p, r, nrhs = 24000, 128, 6, 16, 2
    tol = 1e-12 if precision == "fp64" else 1e-10
    ab = inputs.dominant_band(n, k, 1.1, 88)
    f = inputs.rhs(n, nrhs, 88)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, precision=precision, tol=tol, reduced="truncated",
                        transpose=transpose)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x, trans=transpose)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= tol * 1.01
    if not transpose:
        xs = scipy.linalg.solve_banded((k, k), ab, f)
        assert rel(x, xs) <= 1e4 * tol


def test_wide_convection_diffusion_bicgstab(torch_cuda):
    """2-D convection-diffusion, 96 x 96 grid (k = 96, 5 nonzero diagonals of
    193), Pe = 0.5: mixed TF32 factors with BiCGStab to 1e-10."""
    nx, p, r = 96, 8, 8
    ab = inputs.convection_diffusion_band(nx, 0.5)
    k, n = nx, ab.shape[1]
    f = inputs.rhs(n, 2, 17)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, precision="tf32", tol=1e-10, outer="bicgstab",
                        reduced="truncated", max_iter=200)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= 1.01e-10
