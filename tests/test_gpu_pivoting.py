"""Partial pivoting inside the partitions (pivoting = 1) on the GPU against the
oracle's pivoted factorisation (gbtf2 order, row exchanges within A_i only).

Tolerances as in test_gpu_parity: one FP64 preconditioner application within
1e-12 of the oracle (relative 2-norm); mixed precision within 5e-5; outer
iterations to tol per column, recomputed with the oracle's band product.
The weakly dominant inputs (dominance 0.6) make the diagonal lose the pivot
search in most columns, so the row exchanges are exercised throughout.
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


def gpu_solve(torch, ab, f, k, p, r, transpose=False, allow_unconverged=False, **kw):
    from paper_2504_11167_gb300.solver import LRSpike
    n = ab.shape[1]
    band = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(np.atleast_2d(f.T))).cuda()
    with LRSpike(n, k, p, r, pivoting=True, **kw) as s:
        s.factor(band)
        x, info = (s.solve_transpose if transpose else s.solve)(ft, allow_unconverged=allow_unconverged)
        out = x.cpu().numpy().T.copy()
    return out.reshape(f.shape), info


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # n, k, p, r, dom, compress, reduced, nrhs
    (3000, 16, 4, 4, 0.6, "spike", "full", 1),
    (2000, 5, 3, 2, 0.6, "spike", "full", 2),          # KB = 8, ragged partitions
    (6000, 64, 4, 16, 0.6, "spike", "truncated", 1),   # KB = 64
    (4133, 32, 5, 8, 0.6, "coupling", "full", 3),
    (5000, 24, 6, 6, 0.6, "coupling", "truncated", 2),  # k not a block size
    (70, 16, 4, 3, 0.6, "spike", "full", 1),            # n_i = 17/18 just above k
    (2000, 12, 1, 3, 0.6, "spike", "full", 1),          # p = 1: plain pivoted band solve
    (2000, 12, 4, 0, 0.6, "spike", "full", 1),          # r = 0: block Jacobi
    (1000, 16, 3, 16, 0.6, "spike", "full", 2),         # r = k: exact SPIKE
]


def case_id(c):
    return "n{}-k{}-p{}-r{}-{}-{}-q{}".format(c[0], c[1], c[2], c[3], c[5], c[6], c[7])


@pytest.mark.parametrize("case", CASES, ids=[case_id(c) for c in CASES])
def test_pivoted_preconditioner_parity_fp64(torch_cuda, case):
    n, k, p, r, dom, compress, reduced, nrhs = case
    seed = 1000 + n + k
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, nrhs, seed)
    if nrhs == 1:
        f = f[:, 0]
    fac = O.factor(ab, k, p, r, compress=compress, reduced=reduced, pivoting=True)
    got, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced, outer="none")
    check(got, O.apply(fac, np.asarray(f)), n, p, 1e-12)
    gotT, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced, outer="none",
                        transpose=True)
    check(gotT, O.apply_T(fac, np.asarray(f)), n, p, 1e-12)


@pytest.mark.parametrize("case", CASES[:5], ids=[case_id(c) for c in CASES[:5]])
def test_pivoted_preconditioner_parity_mixed(torch_cuda, case):
    n, k, p, r, dom, compress, reduced, nrhs = case
    seed = 1000 + n + k
    ab = inputs.dominant_band(n, k, dom, seed)
    f = inputs.rhs(n, nrhs, seed)
    fac = O.factor(ab, k, p, r, compress=compress, reduced=reduced, pivoting=True)
    got, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced, outer="none",
                       precision="fp32")
    check(got, O.apply(fac, np.asarray(f)), n, p, MIXED_TOL)
    gotT, _ = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, reduced=reduced, outer="none",
                        precision="fp32", transpose=True)
    check(gotT, O.apply_T(fac, np.asarray(f)), n, p, MIXED_TOL)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
@pytest.mark.parametrize("outer", ["ir", "bicgstab"])
@pytest.mark.parametrize("transpose", [False, True])
def test_pivoted_outer_iteration_reaches_tolerance(torch_cuda, precision, tol, outer, transpose):
    n, k, p, r, nrhs = 20011, 32, 7, 8, 3
    ab = inputs.dominant_band(n, k, 0.6, 55)
    f = inputs.rhs(n, nrhs, 55)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, precision=precision, tol=tol, outer=outer,
                        transpose=transpose, reduced="truncated")
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x, trans=transpose)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= tol * 1.01
    if not transpose:
        xs = scipy.linalg.solve_banded((k, k), ab, f)
        assert rel(x, xs) <= 1e4 * tol


def test_zero_diagonal_needs_pivoting(torch_cuda):
    """A_ii = 0 in two partitions: the unpivoted factorisation stops with
    SINGULAR, the pivoted one solves to 1e-12 like the oracle."""
    from paper_2504_11167_gb300.solver import LRSpike, LRSpikeError
    torch = torch_cuda
    n, k, p, r = 2000, 8, 4, 2
    ab = inputs.dominant_band(n, k, 1.5, 3)
    ab[k, 0] = 0.0
    ab[k, 777] = 0.0
    band = torch.from_numpy(ab).cuda()
    with LRSpike(n, k, p, r) as s:
        with pytest.raises(LRSpikeError) as e:
            s.factor(band)
        assert e.value.name == "SINGULAR"
    f = inputs.rhs(n, 1, 3)
    x, info = gpu_solve(torch, ab, f, k, p, r, tol=1e-12)
    assert info["converged"]
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    assert rel(x, xs) <= 1e-10


def test_pivoted_singular_column_is_reported(torch_cuda):
    from paper_2504_11167_gb300.solver import LRSpike, LRSpikeError
    torch = torch_cuda
    n, k = 600, 4
    ab = inputs.dominant_band(n, k, 0.6, 4)
    for d in range(2 * k + 1):     # column 250 of A is zero
        ab[d, 250] = 0.0
    with LRSpike(n, k, 2, 2, pivoting=True) as s:
        with pytest.raises(LRSpikeError) as e:
            s.factor(torch.from_numpy(ab).cuda())
        assert e.value.name == "SINGULAR" and "row" in str(e.value)
