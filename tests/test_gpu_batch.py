"""Batched uneven systems in one CUDA-graph launch (graph-safe handles on a
pool of streams): every system converges to 1e-10 (FP32 factors, FP64
refinement), replaying the graph reproduces the eager launches bit for bit,
a system whose residual meets tol skips its remaining steps on the device,
and the autotuner returns a shape that solves its class."""
import numpy as np
import pytest
import scipy.linalg

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


def make_systems(torch, count, seed):
    rng = np.random.default_rng(seed)
    out, host = [], []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(3000), np.log(40000)))))
        k = int(rng.choice([8, 16, 32, 64]))
        ab = inputs.dominant_band(n, k, 1.5, seed + i)
        f = inputs.rhs(n, 1, seed + i)[:, 0]
        out.append((torch.from_numpy(ab).cuda(), torch.from_numpy(f).cuda(), k))
        host.append((ab, f, k))
    return out, host


def test_graph_batch_converges_and_matches_eager(torch_cuda):
    torch = torch_cuda
    from paper_2504_11167_gb300.batch import BatchSolver
    systems, host = make_systems(torch, 12, 700)
    b = BatchSolver(systems, iterations=8, streams=4)
    b.run_eager()
    torch.cuda.synchronize()
    eager = [x.clone() for x in b.x]
    for info in b.finish():
        assert info["converged"] and info["max_rel_residual"] <= 1e-10
    b.capture()
    for x in b.x:
        x.zero_()
    b.replay()
    infos = b.finish()
    for (ab, f, k), x, xe, info in zip(host, b.x, eager, infos):
        assert info["converged"]
        assert torch.equal(x, xe)                    # same kernels, same order: bitwise
        xs = scipy.linalg.solve_banded((k, k), ab, f)
        xg = x[0].cpu().numpy()
        assert np.linalg.norm(xg - xs) <= 1e-8 * np.linalg.norm(xs)
    b.close()


def test_autotune_picks_a_working_candidate(torch_cuda):
    torch = torch_cuda
    from paper_2504_11167_gb300 import batch
    n, k = 20000, 16
    ab = inputs.dominant_band(n, k, 1.5, 9)
    f = inputs.rhs(n, 1, 9)[:, 0]
    band, ft = torch.from_numpy(ab).cuda(), torch.from_numpy(f).cuda()
    best = batch.autotune({(k, batch.size_class(n)): (band, ft)}, iterations=8, reps=2)
    shape = best[(k, batch.size_class(n))]
    assert shape in batch.candidate_shapes(n, k)
    b = batch.BatchSolver([(band, ft, k)], shapes=[shape], iterations=8, streams=1)
    b.run_eager()
    assert b.finish()[0]["converged"]
    b.close()


def test_graph_safe_refinement_exits_on_the_device(torch_cuda):
    """A graph-safe IR solve enqueues max_iter steps; the residual that meets
    tol raises the handle's device flag and the remaining steps return at
    entry.  The reported step count equals the host-driven IR's, x equals (bit
    for bit) the x of a graph-safe solve enqueued with exactly that many
    steps, and an unreachable tol (0) runs every step."""
    torch = torch_cuda
    from paper_2504_11167_gb300.solver import LRSpike
    n, k, p, r = 30000, 16, 6, 4
    ab = inputs.dominant_band(n, k, 1.5, 77)
    f = inputs.rhs(n, 1, 77)
    band = torch.from_numpy(ab).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(f.T)).cuda()

    def graph_safe(max_iter, tol):
        with LRSpike(n, k, p, r, precision="fp32", reduced="truncated", outer="ir", tol=tol,
                     max_iter=max_iter, max_nrhs=1, graph_safe=True) as s:
            s.factor(band)
            x = torch.empty_like(ft)
            s.solve(ft, x)
            info = s.finish(nrhs=1, allow_unconverged=True)
        return x, info

    x30, i30 = graph_safe(30, 1e-10)
    assert i30["converged"] and 1 <= i30["iterations"] < 30
    with LRSpike(n, k, p, r, precision="fp32", reduced="truncated", outer="ir", tol=1e-10, max_iter=30) as s:
        s.factor(band)
        _, ih = s.solve(ft)
    assert ih["iterations"] == i30["iterations"]
    xe, ie = graph_safe(i30["iterations"], 1e-10)
    assert ie["converged"] and ie["iterations"] == i30["iterations"]
    assert torch.equal(x30, xe)
    assert ie["max_rel_residual"] == i30["max_rel_residual"]
    x0, i0 = graph_safe(5, 0.0)
    assert not i0["converged"] and i0["iterations"] == 5


def test_graph_replays_reset_the_exit_flag(torch_cuda):
    """Each replay clears the flag before its first residual: a batch replayed
    twice reports the same step counts and the same x."""
    torch = torch_cuda
    from paper_2504_11167_gb300.batch import BatchSolver
    systems, _ = make_systems(torch, 6, 900)
    b = BatchSolver(systems, iterations=12, streams=3)
    b.capture()
    b.replay()
    first = b.finish()
    x1 = [x.clone() for x in b.x]
    for x in b.x:
        x.fill_(float("nan"))
    b.replay()
    second = b.finish()
    assert [i["iterations"] for i in first] == [i["iterations"] for i in second]
    assert all(i["converged"] and i["iterations"] < 12 for i in second)
    for a, c in zip(x1, b.x):
        assert torch.equal(a, c)
    b.close()


@pytest.mark.parametrize("pivoting,transpose,nrhs", [(False, True, 1), (True, False, 1), (True, True, 1),
                                                     (False, False, 3), (False, True, 3)])
def test_graph_safe_exit_on_every_kernel_path(torch_cuda, pivoting, transpose, nrhs):
    """The early exit on the other kernels a graph-safe step runs: the
    transposed D-stage, the pivoted D-stages, the multi-column retrieval.  A
    solve enqueued with 40 steps equals, bit for bit, one enqueued with
    exactly the steps it reports, and every column meets tol."""
    torch = torch_cuda
    from paper_2504_11167_gb300.solver import LRSpike
    n, k, p, r = 24000, 16, 6, 4
    ab = inputs.dominant_band(n, k, 0.8 if pivoting else 1.5, 91)
    f = inputs.rhs(n, nrhs, 91)
    band = torch.from_numpy(ab).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(f.T)).cuda()

    def graph_safe(max_iter):
        with LRSpike(n, k, p, r, precision="fp32", reduced="truncated", outer="ir", tol=1e-10,
                     max_iter=max_iter, max_nrhs=nrhs, pivoting=pivoting, graph_safe=True) as s:
            s.factor(band)
            x = torch.empty_like(ft)
            (s.solve_transpose if transpose else s.solve)(ft, x)
            info = s.finish(nrhs=nrhs, allow_unconverged=True)
        return x, info

    x40, i40 = graph_safe(40)
    assert i40["converged"] and 1 <= i40["iterations"] < 40
    assert max(i40["rel_residual"][:nrhs]) <= 1e-10
    xe, ie = graph_safe(i40["iterations"])
    assert ie["iterations"] == i40["iterations"]
    assert torch.equal(x40, xe)
