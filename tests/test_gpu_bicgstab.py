"""BiCGStab outer iteration on the GPU (right-preconditioned, FP64 vectors)
against the oracle's BiCGStab and against the plain definition x = A^{-1} f.

Tolerances: relative residual <= tol per column (1e-12 FP64, 1e-10 mixed),
recomputed here with the oracle's FP64 band product; the forward error against
LAPACK's banded solve <= 1e3 tol (the test matrices have kappa well below 1e3).
Iteration counts: the GPU runs the same recurrence as the oracle in FP64, with
sums added in a different order, so the counts agree to within two.
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


def relres(ab, k, x, f, transpose=False):
    res = np.asarray(f) - O.band_matvec(ab, k, x, trans=transpose)
    return np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)


def test_bicgstab_converges_where_ir_stalls(torch_cuda):
    """2-D convection-diffusion (nx = 48, Pe = 0.5, k = 48), p = 16, r = 2,
    truncated reduced system: the oracle's IR stalls near 1e-7, BiCGStab reaches
    1e-12.  The GPU path shows the same split."""
    torch = torch_cuda
    nx, p, r = 48, 16, 2
    ab = inputs.convection_diffusion_band(nx, 0.5)
    k, n = nx, ab.shape[1]
    f = inputs.rhs(n, 2, 5)
    fac = O.factor(ab, k, p, r, reduced="truncated")
    ref = O.bicgstab(ab, k, fac, f, tol=1e-12, max_iter=100)
    assert ref.converged
    x, info = gpu_solve(torch, ab, f, k, p, r, reduced="truncated", outer="bicgstab", tol=1e-12, max_iter=100)
    assert info["converged"]
    assert relres(ab, k, x, f).max() <= 1e-12
    assert abs(info["iterations"] - ref.iterations) <= 2
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-9
    _, info_ir = gpu_solve(torch, ab, f, k, p, r, reduced="truncated", outer="ir", tol=1e-12,
                           allow_unconverged=True)
    assert not info_ir["converged"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("reduced", ["full", "truncated"])
def test_bicgstab_reaches_tolerance(torch_cuda, precision, tol, transpose, reduced):
    n, k, p, r, nrhs = 20011, 32, 7, 4, 3
    ab = inputs.dominant_band(n, k, 0.9, 41)
    f = inputs.rhs(n, nrhs, 41)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, reduced=reduced, precision=precision, tol=tol,
                        outer="bicgstab", transpose=transpose)
    assert info["converged"] and info["iterations"] >= 1
    rr = relres(ab, k, x, f, transpose)
    assert rr.max() <= tol * 1.01
    # the reported residual is the GPU's own f - A x; the two differ by the
    # rounding of a residual computation, ~1e-16 relative to |A| |x| / |f|
    assert np.allclose(info["rel_residual"], rr, rtol=1e-2, atol=1e-15)
    if precision == "fp64" and not transpose:
        fac = O.factor(ab, k, p, r, reduced=reduced)
        ref = O.bicgstab(ab, k, fac, f, tol=tol)
        assert abs(info["iterations"] - ref.iterations) <= 2


def test_bicgstab_zero_column_and_iteration_limit(torch_cuda):
    """A zero right-hand side column stays x = 0 while the others iterate; a
    limit of one iteration ends with NOT_CONVERGED and the last iterate."""
    from paper_2504_11167_gb300.solver import LRSpikeError
    n, k, p, r = 9001, 16, 4, 2
    ab = inputs.dominant_band(n, k, 1.1, 12)
    f = inputs.rhs(n, 3, 12)
    f[:, 1] = 0.0
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, outer="bicgstab", tol=1e-12)
    assert info["converged"] and np.all(x[:, 1] == 0.0)
    assert relres(ab, k, x[:, [0, 2]], f[:, [0, 2]]).max() <= 1e-12
    with pytest.raises(LRSpikeError) as e:
        gpu_solve(torch_cuda, ab, f, k, p, r, outer="bicgstab", tol=1e-14, max_iter=1)
    assert e.value.name == "NOT_CONVERGED"
    x1, info1 = gpu_solve(torch_cuda, ab, f, k, p, r, outer="bicgstab", tol=1e-14, max_iter=1,
                          allow_unconverged=True)
    assert info1["iterations"] == 1 and 0 < info1["max_rel_residual"] < 1e-2
