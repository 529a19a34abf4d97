"""Batched uneven systems in one CUDA-graph launch (graph-safe handles on a
pool of streams): every system converges to 1e-10 (FP32 factors, FP64
refinement), replaying the graph reproduces the eager launches bit for bit,
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
