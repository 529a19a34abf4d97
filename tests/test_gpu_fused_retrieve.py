"""The IR loop's fused retrieval + residual (one right-hand side, unpivoted
k <= 64 factors, every partition holding >= 256 + 2k rows): the retrieval
x += |r| (g - U z) of an application is formed by the next residual kernel,
the iterate alternating between the caller's buffer and a second one.

* Bit-identical to the separate kernels: a graph-safe handle with an
  unreachable tol runs exactly max_iter unfused steps (residual, D-stage, reduced solve, retrieval), the
  same arithmetic in the same order; after the same number of steps the two
  iterates agree bit for bit, for an even and an odd step count (the fused
  loop's result then sits in one or the other buffer).
* The fused solve reaches the tolerance (residual recomputed with the oracle's
  FP64 band product) and agrees with LAPACK's banded solve.
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


# n, k, p, r, compression: ragged n (n mod p != 0, n mod 256 != 0)
CASES = [(20011, 16, 8, 4, "coupling"), (40037, 64, 8, 16, "coupling"), (30001, 32, 6, 8, "spike")]


def run_pair(torch, case, precision, steps):
    from paper_2504_11167_gb300.solver import LRSpike
    n, k, p, r, comp = case
    seed = 500 + k
    band = torch.from_numpy(inputs.dominant_band(n, k, 1.1, seed)).cuda()
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, 1, seed)[:, 0])).cuda()
    with LRSpike(n, k, p, r, precision=precision, compress=comp, tol=1e-300, max_iter=steps) as s:
        s.factor(band)
        xf, info = s.solve(f, allow_unconverged=True)
        xf = xf.clone()
    with LRSpike(n, k, p, r, precision=precision, compress=comp, tol=1e-300, max_iter=steps,
                 graph_safe=True) as s:
        s.factor(band)
        xg, _ = s.solve(f)
        s.finish(nrhs=1, allow_unconverged=True)
        xg = xg.clone()
    return xf, xg, info


@pytest.mark.parametrize("steps", [2, 3])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{}-k{}-p{}-{}".format(c[0], c[1], c[2], c[4]))
def test_fused_equals_separate_kernels_bitwise(torch_cuda, case, precision, steps):
    xf, xg, info = run_pair(torch_cuda, case, precision, steps)
    assert info["iterations"] == steps
    assert torch_cuda.equal(xf, xg)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-10), ("fp64", 1e-12)])
def test_fused_solve_reaches_tolerance(torch_cuda, precision, tol):
    from paper_2504_11167_gb300.solver import LRSpike
    n, k, p, r = 50021, 64, 10, 16
    ab = inputs.dominant_band(n, k, 1.1, 901)
    f = inputs.rhs(n, 1, 901)[:, 0]
    band = torch_cuda.from_numpy(ab).cuda()
    with LRSpike(n, k, p, r, precision=precision, compress="coupling", tol=tol) as s:
        s.factor(band)
        x, info = s.solve(torch_cuda.from_numpy(np.ascontiguousarray(f)).cuda())
        x = x.cpu().numpy()
    assert info["converged"]
    res = f - O.band_matvec(ab, k, x)
    assert np.linalg.norm(res) / np.linalg.norm(f) <= tol * 1.01
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e3 * tol
