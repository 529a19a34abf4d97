"""Wide bands (64 < k <= 1024) on the GPU: blocks of W = 64 ceil(k/64), block
products batched over the partitions (SIMT GEMMs in FP64 / FP32, tcgen05
tensor cores with TF32 or BF16 operands), the randomized truncation of the
spikes by the HMT proto-algorithm on each spike, the cluster D-stage.

Parity: one FP64 preconditioner application against the oracle with the same
randomized truncation (same sketches: SplitMix64 + Box-Muller, seeds
0x4C52535049 + 2i + side, ell = 2r, two power passes).  The oracle
orthonormalises with Householder QR, the GPU with shifted CholeskyQR3; both
span the same range to rounding, so the bound is the FP64 one-application
bound of the narrow path, 1e-12 (2-norm), 1e-11 per partition (max-norm).
Mixed FP32 / TF32 / BF16 solves: relative residual <= 1e-10 per column (IR,
or BiCGStab where IR stalls), recomputed with the oracle's FP64 band product.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs
from _parity import check, rel

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


CASES = [
    # n, k, p, r, dom, reduced, nrhs
    (6000, 96, 4, 8, 1.2, "truncated", 1),     # W = 128
    (5000, 70, 3, 6, 1.3, "full", 2),          # W = 128 > k, ragged partitions
    (20000, 200, 5, 16, 1.1, "truncated", 3),  # W = 256: two levels of recursive halving
    (9000, 130, 3, 10, 1.2, "full", 5),        # W = 192: unequal split 128 + 64, nrhs > 4
    (3000, 100, 1, 4, 1.5, "full", 1),         # p = 1: the wide band LU alone
    (6200, 1024, 3, 16, 1.1, "truncated", 4),  # W = 1024: the convection-diffusion block size
    (8000, 96, 3, 8, 1.2, "truncated", 16),    # widest nrhs: four D-stage column chunks
]


def case_id(c):
    return "n{}-k{}-p{}-r{}-{}-q{}".format(c[0], c[1], c[2], c[3], c[5], c[6])


@pytest.mark.parametrize("case", CASES, ids=[case_id(c) for c in CASES])
def test_wide_preconditioner_parity_fp64(torch_cuda, case):
    n, k, p, r, dom, reduced, nrhs = case
    seed = 2000 + n + k
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, nrhs, seed)
    fac = O.factor(ab, k, p, r, reduced=reduced, threads=p)   # k > 64: randomized truncation
    got, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, outer="none")
    check(got, O.apply(fac, np.asarray(f)), n, p, 1e-12)
    gotT, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, outer="none", transpose=True)
    check(gotT, O.apply_T(fac, np.asarray(f)), n, p, 1e-12)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16", "fp64"])
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


@pytest.mark.parametrize("precision,bound,n,k", [("tf32", 2e-3, 12000, 128), ("bf16", 3e-2, 12000, 128),
                                                 ("tf32", 2e-3, 40000, 520), ("bf16", 3e-2, 40000, 520)])
def test_wide_tensor_core_preconditioner_error(torch_cuda, precision, bound, n, k):
    """One application with tensor-core block products against the FP64
    oracle.  TF32 keeps 10 mantissa bits (unit roundoff 2^-11 = 4.9e-4), BF16
    7 (2^-8 = 3.9e-3); the rounding of the operands of a product of order W
    enters M^{-1} f relatively at a few units of that roundoff through the
    well-conditioned block chain of a dominant band, so the bounds are four
    (TF32) and eight (BF16) times the operand roundoff.  With BF16 factors the
    D-stage also reads BF16 tiles: one more rounding of the same size per
    product.  k = 520 (W = 576): D-stage boxes of 256 columns, three per line."""
    p, r = 4, 16
    ab = inputs.dominant_band(n, k, 1.2, 31)
    f = inputs.rhs(n, 2, 31)
    fac = O.factor(ab, k, p, r, reduced="truncated")
    got, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced="truncated", outer="none", precision=precision)
    assert rel(got, O.apply(fac, np.asarray(f))) <= bound


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_wide_convection_diffusion_bicgstab(torch_cuda, precision):
    """2-D convection-diffusion, 96 x 96 grid (k = 96, 5 nonzero diagonals of
    193), Pe = 0.5: tensor-core factors with BiCGStab to 1e-10."""
    nx, p, r = 96, 8, 8
    ab = inputs.convection_diffusion_band(nx, 0.5)
    k, n = nx, ab.shape[1]
    f = inputs.rhs(n, 2, 17)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, precision=precision, tol=1e-10, outer="bicgstab",
                        reduced="truncated", max_iter=200)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= 1.01e-10


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_wide_rank64(torch_cuda, precision):
    """r = 64 (reduced-system blocks of 128 x 128, inverted in place; sketches
    of ell = 128 columns): one application within the tensor-core bound of the
    FP64 oracle, and the refinement to 1e-10."""
    n, k, p, r = 20000, 192, 4, 64
    ab = inputs.dominant_band(n, k, 1.2, 41)
    f = inputs.rhs(n, 3, 41)  # three columns: the multi-column retrieval over 128 low-rank columns
    fac = O.factor(ab, k, p, r, reduced="truncated", threads=p)
    got, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced="truncated", outer="none", precision=precision)
    assert rel(got, O.apply(fac, np.asarray(f))) <= (2e-3 if precision == "tf32" else 3e-2)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, reduced="truncated", precision=precision, tol=1e-10)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= 1.01e-10
