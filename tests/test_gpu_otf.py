"""LR-SPIKE-OTF on the GPU (reduced = "otf"): the true reduced system on the
interface tips, solved by right-preconditioned BiCGStab with on-the-fly spike
products (one D-stage each) and the truncated low-rank preconditioner.

Parity with the oracle (same algorithm, FP64):
  * one OTF solve (outer "none") with a tight reduced tolerance reproduces
    x = A^{-1} f (LAPACK banded solve) and the oracle's OTF result to 1e-9;
  * the reduced BiCGStab takes about as many iterations as the oracle's
    (within 2: the two run the same recurrences, rounding differs);
  * with the default reduced tolerance 1e-8 one OTF solve is accurate to
    about 1e-8, so refinement around it converges in 2-3 outer steps (FP64 to
    1e-12, mixed FP32 + FP64 to 1e-10; residuals recomputed with the oracle).
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


def gpu_solve(torch, ab, f, k, p, r, **kw):
    from paper_2504_11167_gb300.solver import LRSpike
    n = ab.shape[1]
    band = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(np.atleast_2d(f.T))).cuda()
    with LRSpike(n, k, p, r, reduced="otf", **kw) as s:
        s.factor(band)
        x, info = s.solve(ft)
        out = x.cpu().numpy().T.copy()
    return out.reshape(f.shape), info


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # n, k, p, r, dom, compress, nrhs
    (6000, 8, 6, 3, 1.2, "spike", 1),
    (5000, 16, 5, 4, 1.1, "coupling", 2),
    (9000, 64, 4, 16, 1.1, "coupling", 1),
    (420, 40, 5, 6, 1.3, "spike", 3),      # n_i = 84 < 2k: the two tips of a partition overlap
    (6000, 96, 4, 8, 1.2, "spike", 2),     # wide band (W = 128): solves on the wide-band factors
]


def case_id(c):
    return "n{}-k{}-p{}-r{}-{}-q{}".format(c[0], c[1], c[2], c[3], c[5], c[6])


@pytest.mark.parametrize("case", CASES, ids=[case_id(c) for c in CASES])
def test_one_otf_solve_matches_oracle_and_exact_solution(torch_cuda, case):
    n, k, p, r, dom, compress, nrhs = case
    ab = inputs.dominant_band(n, k, dom, 3000 + n + k)
    f = inputs.rhs(n, nrhs, 3000 + n + k)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, compress=compress, outer="none", otf_tol=1e-12,
                        otf_max_iter=200)
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    assert rel(x, xs) <= 1e-9
    fac = O.factor(ab, k, p, r, compress=compress, reduced="truncated")
    xo, its = O.otf_apply(fac, ab, np.asarray(f), otf_tol=1e-12, max_iter=200)
    assert rel(x, xo) <= 1e-9
    assert abs(info["reduced_iterations"] - its) <= 2, (info["reduced_iterations"], its)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
def test_otf_with_refinement_reaches_tolerance(torch_cuda, precision, tol):
    n, k, p, r = 40000, 32, 8, 8
    ab = inputs.dominant_band(n, k, 1.05, 77)
    f = inputs.rhs(n, 2, 77)
    x, info = gpu_solve(torch_cuda, ab, f, k, p, r, precision=precision, tol=tol, compress="coupling")
    assert info["converged"] and info["iterations"] <= 4
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(f, axis=0)).max() <= tol * 1.01
    assert info["reduced_iterations"] >= 1


def test_otf_needs_fewer_outer_steps_than_the_truncated_preconditioner(torch_cuda):
    """The true reduced system: one outer step of OTF does the work of several
    steps of LR-SPIKE-T on a weakly dominant band with a small rank."""
    from paper_2504_11167_gb300.solver import LRSpike
    torch = torch_cuda
    n, k, p, r = 30000, 16, 10, 2
    ab = inputs.dominant_band(n, k, 1.02, 88)
    f = inputs.rhs(n, 1, 88)
    _, i_otf = gpu_solve(torch, ab, f, k, p, r, tol=1e-12)
    band = torch.from_numpy(ab).cuda()
    with LRSpike(n, k, p, r, reduced="truncated", tol=1e-12) as s:
        s.factor(band)
        _, i_t = s.solve(torch.from_numpy(np.ascontiguousarray(f.T)).cuda())
    assert i_otf["converged"] and i_t["converged"]
    assert i_otf["iterations"] < i_t["iterations"]


def test_otf_wide_convection_diffusion(torch_cuda):
    """LR-SPIKE-OTF on a wide, sparse-in-band system (the paper's setting for
    it): 2-D convection-diffusion on a 96 x 96 grid (k = 96), TF32 factors,
    the reduced system iterated to 1e-8 inside FP64 refinement to 1e-10."""
    ab = inputs.convection_diffusion_band(96, 0.5)
    k, n = 96, ab.shape[1]
    f = inputs.rhs(n, 1, 23)
    x, info = gpu_solve(torch_cuda, ab, f, k, 8, 8, precision="tf32", tol=1e-10, max_iter=20)
    assert info["converged"]
    res = np.asarray(f) - O.band_matvec(ab, k, x)
    assert np.linalg.norm(res) / np.linalg.norm(f) <= 1.01e-10
