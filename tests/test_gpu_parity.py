"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (each also checked per partition in the max-norm at ten times
the bound, tests/_parity.py):
  FP64, one preconditioner application: ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-12.
  Mixed (FP32 working precision), one application: <= 5e-5.  Derivation: the
    FP32 unit roundoff is 6e-8; a block sweep over a partition accumulates
    O(KB) rounding steps per row through a well-conditioned chain (dominant
    A_i, kappa of a few), the Gram/Jacobi subspace carries ~1e-6 relative
    error for singular-value gaps of >= 10 %, giving ~1e-5 in the worst
    component of M^{-1} f; 5e-5 leaves a factor of a few.
  Outer iterations: relative residual <= tol per column (1e-12 FP64, 1e-10 mixed),
    recomputed here with the oracle's FP64 band product.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs
from _parity import check

pytestmark = pytest.mark.gpu

MIXED_TOL = 5e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def gpu_solve(torch, ab, f, k, p, r, transpose=False, host=False, **kw):
    from paper_2504_11167_gb300.solver import LRSpike
    n = ab.shape[1]
    dev = "cpu" if host else "cuda"
    band = torch.from_numpy(np.ascontiguousarray(ab)).to(dev)
    F = np.ascontiguousarray(np.atleast_2d(f.T))      # (nrhs, n): row q = column q
    ft = torch.from_numpy(F).to(dev)
    with LRSpike(n, k, p, r, **kw) as s:
        s.factor(band)
        x, info = (s.solve_transpose if transpose else s.solve)(ft)
        out = x.cpu().numpy().T.copy()
        sig, _ = s.reduced()
    return out.reshape(f.shape), info, sig


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # n, k, p, r, dom, compress, reduced, nrhs
    (1000, 5, 3, 2, 1.5, "spike", "full", 1),           # KB = 8, ragged partitions
    (4133, 16, 4, 4, 1.5, "spike", "truncated", 2),
    (4133, 16, 4, 4, 1.5, "coupling", "full", 1),
    (3000, 32, 5, 8, 1.2, "spike", "full", 3),
    (6000, 64, 6, 16, 1.1, "spike", "truncated", 1),
    (6000, 64, 6, 16, 1.1, "coupling", "truncated", 5),
    (7000, 64, 5, 32, 1.1, "spike", "full", 4),
    (2000, 12, 1, 3, 1.5, "spike", "full", 1),          # p = 1: plain band solve
    (2000, 12, 4, 0, 1.5, "spike", "full", 1),          # r = 0: block Jacobi
    (2000, 12, 4, 12, 1.5, "spike", "full", 2),         # r = k: exact SPIKE
    (600, 20, 2, 7, 1.3, "spike", "truncated", 1),      # p = 2
    (70, 16, 4, 3, 1.5, "spike", "full", 1),            # n_i = 17/18 just above k
    (260, 33, 3, 5, 1.4, "coupling", "full", 2),        # k not a block size
    (50000, 8, 16, 4, 1.5, "spike", "truncated", 16),   # many blocks, widest nrhs
    (5000, 24, 4, 6, 1.3, "coupling", "full", 1),       # KB = 32, one column: warp D-stage
    (9000, 40, 3, 10, 1.2, "spike", "truncated", 1),    # KB = 64, one column: warp D-stage
    (12800, 8, 64, 4, 1.2, "spike", "full", 2),         # FULL by cyclic reduction: 63 interfaces, 6 levels
    (6600, 12, 33, 5, 1.3, "coupling", "full", 1),      # 32 interfaces: the last level keeps one block
]


def case_id(c):
    return "n{}-k{}-p{}-r{}-{}-{}-q{}".format(c[0], c[1], c[2], c[3], c[5], c[6], c[7])


@pytest.mark.parametrize("case", CASES, ids=[case_id(c) for c in CASES])
def test_preconditioner_parity_fp64(torch_cuda, case):
    n, k, p, r, dom, compress, reduced, nrhs = case
    seed = 1000 + n + k + r
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, nrhs, seed)
    fac = O.factor(ab, k, p, r, compress=compress, reduced=reduced)
    want = O.apply(fac, np.asarray(f))
    got, _, sig = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced,
                            outer="none", precision="fp64")
    check(got, want, n, p, 1e-12)
    if r == k and reduced == "full":
        assert rel(got, scipy.linalg.solve_banded((k, k), ab, f)) <= 1e-11
    # kept singular values (unique, unlike the singular vectors); the Gram
    # route resolves sigma_j to ~eps sigma_1^2 / sigma_j, so compare against sigma_1
    for i in range(p):
        for side, sv in ((0, fac.sigV[i] if i < p - 1 else None), (1, fac.sigW[i] if i > 0 else None)):
            if sv is None or r == 0:
                continue
            kept = np.where(sv[:r] > 1e-13 * sv[0], sv[:r], 0.0)
            assert np.allclose(sig[i, side], kept, rtol=0, atol=1e-9 * sv[0])
    # transposed operator
    gotT, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced,
                           outer="none", precision="fp64", transpose=True)
    check(gotT, O.apply_T(fac, np.asarray(f)), n, p, 1e-12)


@pytest.mark.parametrize("case", CASES[:7], ids=[case_id(c) for c in CASES[:7]])
def test_preconditioner_parity_mixed(torch_cuda, case):
    n, k, p, r, dom, compress, reduced, nrhs = case
    seed = 2000 + n + k
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, nrhs, seed)
    fac = O.factor(ab, k, p, r, compress=compress, reduced=reduced)
    got, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced,
                          outer="none", precision="fp32")
    check(got, O.apply(fac, np.asarray(f)), n, p, MIXED_TOL)
    gotT, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced,
                           outer="none", precision="fp32", transpose=True)
    check(gotT, O.apply_T(fac, np.asarray(f)), n, p, MIXED_TOL)


# FP32, KB = 64, COUPLING with 2r <= 32: the balanced spike sweep writes the
# u-factors into Ucat itself.  r < 16 leaves padding columns in the 32-column
# panel (T half: columns r..15, W half: 16+r..31); with p = 2 the first
# partition has no W spike and the last no T spike (their u columns are zero).
SWEEP_U_CASES = [(6000, 50, 5, 12, 1.2), (3000, 64, 2, 9, 1.2), (8000, 64, 4, 16, 1.1)]


@pytest.mark.parametrize("case", SWEEP_U_CASES, ids=["n{}-k{}-p{}-r{}".format(*c[:4]) for c in SWEEP_U_CASES])
def test_coupling_u_factors_written_by_the_sweep(torch_cuda, case):
    n, k, p, r, dom = case
    seed = 3000 + n + k + r
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, 1, seed)
    fac = O.factor(ab, k, p, r, compress="coupling", reduced="truncated")
    got, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress="coupling", reduced="truncated",
                          outer="none", precision="fp32")
    check(got, O.apply(fac, np.asarray(f)), n, p, MIXED_TOL)
    x, info, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress="coupling", precision="fp32", tol=1e-10)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert np.linalg.norm(res) / np.linalg.norm(f) <= 1e-10 * 1.01


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
@pytest.mark.parametrize("reduced", ["full", "truncated"])
@pytest.mark.parametrize("transpose", [False, True])
def test_outer_iteration_reaches_tolerance(torch_cuda, precision, tol, reduced, transpose):
    n, k, p, r, nrhs = 20011, 32, 7, 6, 3
    ab = inputs.dominant_band(n, k, 1.1, 77)
    f = inputs.rhs(n, nrhs, 77)
    x, info, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, precision=precision,
                           tol=tol, transpose=transpose)
    assert info["converged"] and info["iterations"] >= 1
    res = np.asarray(f) - O.band_matvec(ab, k, x, trans=transpose)
    relres = np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)
    assert relres.max() <= tol * 1.01
    abT = ab if not transpose else None
    if not transpose:
        xs = scipy.linalg.solve_banded((k, k), abT, f)
        assert rel(x, xs) <= 1e3 * tol


def test_host_buffers_match_device_buffers(torch_cuda):
    n, k, p, r = 9000, 16, 5, 4
    ab = inputs.dominant_band(n, k, 1.2, 5)
    f = inputs.rhs(n, 2, 5)
    a, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, precision="fp32")
    b, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, precision="fp32", host=True)
    assert np.array_equal(a, b)


def test_repeat_solves_are_bitwise_identical(torch_cuda):
    from paper_2504_11167_gb300.solver import LRSpike
    torch = torch_cuda
    n, k, p, r = 30000, 64, 4, 16
    ab = inputs.dominant_band(n, k, 1.1, 8)
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, 1, 8)[:, 0])).cuda()
    with LRSpike(n, k, p, r, precision="fp32", reduced="truncated") as s:
        s.factor(torch.from_numpy(ab).cuda())
        x1, _ = s.solve(f)
        x1 = x1.clone()
        s.factor(torch.from_numpy(ab).cuda())
        x2, _ = s.solve(f)
    assert torch.equal(x1, x2)


def test_solve_before_factor_and_singular_pivot(torch_cuda):
    from paper_2504_11167_gb300.solver import LRSpike, LRSpikeError
    torch = torch_cuda
    n, k = 500, 4
    ab = inputs.dominant_band(n, k, 1.5, 3)
    with LRSpike(n, k, 2, 2) as s:
        with pytest.raises(LRSpikeError) as e:
            s.solve(torch.zeros(n, dtype=torch.float64, device="cuda"))
        assert e.value.name == "STATE"
        bad = ab.copy()
        bad[:, 100] = 0.0                      # column 100 of A is zero
        with pytest.raises(LRSpikeError) as e:
            s.factor(torch.from_numpy(bad).cuda())
        assert e.value.name == "SINGULAR" and "row" in str(e.value)
        s.factor(torch.from_numpy(ab).cuda())  # recovers after a good factor
        x, info = s.solve(torch.ones(n, dtype=torch.float64, device="cuda"))
        assert info["converged"]


def test_config1_full_size_fp64(torch_cuda):
    """n = 65536, k = 16, p = 8, r = 4, FP64: one application against the
    oracle and the IR solve to 1e-12."""
    n, k, p, r = 65536, 16, 8, 4
    seed = inputs.SEED_BASE + 1
    ab = inputs.dominant_band(n, k, 1.5, seed)
    f = inputs.rhs(n, 1, seed)
    for reduced in ("full", "truncated"):
        fac = O.factor(ab, k, p, r, reduced=reduced)
        got, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, outer="none")
        check(got, O.apply(fac, np.asarray(f)), n, p, 1e-12)
        x, info, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, tol=1e-12)
        res = np.asarray(f) - O.band_matvec(ab, k, x)
        assert np.linalg.norm(res) / np.linalg.norm(f) <= 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
@pytest.mark.parametrize("compress", ["spike", "coupling"])
def test_single_column_solves_k64(torch_cuda, precision, tol, compress):
    """One right-hand side with 64-row blocks (the one-warp-per-partition
    D-stage): the IR solve reaches tol and matches LAPACK's banded solve."""
    n, k, p, r = 40000, 64, 8, 16
    ab = inputs.dominant_band(n, k, 1.1, 19)
    f = inputs.rhs(n, 1, 19)[:, 0]
    x, info, _ = gpu_solve(torch_cuda, ab, f, k, p, r, reduced="truncated", precision=precision, tol=tol,
                           compress=compress)
    assert info["converged"]
    res = f - O.band_matvec(ab, k, x)
    assert np.linalg.norm(res) / np.linalg.norm(f) <= tol * 1.01
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    assert rel(x, xs) <= 1e3 * tol


@pytest.mark.parametrize("compress", ["spike", "coupling"])
def test_tf32_band_lu(torch_cuda, compress):
    """MIXED_TF32 with k <= 64: the band LU's block products on the tensor
    cores.  One application: TF32 operands carry a relative rounding of
    2^-11 = 4.9e-4 into the products; through a well-conditioned chain that
    stays well below 1e-3 of |M^{-1} f| (the FP32 bound is 5e-5).  The FP64
    refinement still reaches 1e-10."""
    n, k, p, r = 6000, 64, 6, 16
    ab = inputs.dominant_band(n, k, 1.1, 5)
    f = inputs.rhs(n, 2, 5)
    fac = O.factor(ab, k, p, r, compress=compress, reduced="truncated")
    got, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced="truncated", outer="none",
                          precision="tf32")
    check(got, O.apply(fac, np.asarray(f)), n, p, 1e-3)
    x, info, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced="truncated", precision="tf32",
                           tol=1e-10)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= 1.01e-10


@pytest.mark.parametrize("precision,tol", [("fp32", MIXED_TOL), ("fp64", 1e-12)])
def test_bench_partition_geometry(torch_cuda, precision, tol):
    """The large banded workload's partition shape: n_i = 16,384 rows, k = 64,
    r = 16, COUPLING compression, TRUNCATED reduced system, p = 8 (n = 131,072),
    so the column band LU, the balanced spike sweep and the D-stage run their
    full-length chains.  One application against the oracle (2-norm and
    per-partition max-norm), then the IR solve, whose refinement steps fuse
    each retrieval into the next residual (mixed mode), to its tolerance."""
    n, k, p, r = 8 * 16384, 64, 8, 16
    seed = inputs.SEED_BASE + 2
    ab = inputs.dominant_band(n, k, 1.1, seed)
    f = inputs.rhs(n, 1, seed)
    fac = O.factor(ab, k, p, r, compress="coupling", reduced="truncated", threads=8)
    got, _, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress="coupling", reduced="truncated", outer="none",
                          precision=precision)
    check(got, O.apply(fac, np.asarray(f)), n, p, tol)
    ir_tol = 1e-12 if precision == "fp64" else 1e-10
    x, info, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress="coupling", reduced="truncated",
                           precision=precision, tol=ir_tol)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert np.linalg.norm(res) / np.linalg.norm(f) <= ir_tol * 1.01
