"""Factorisation of a band held in host memory.  For the column-kernel band
LU (k <= 64, unpivoted, FP32 or FP64 working precision) the upload runs in
partition groups on its own stream, the interface columns first for the
coupling branch, and every group's band LU starts when its columns land.
The kernels and their order within a partition are those of one LU launch
over all partitions (a device band; a profiling handle also uploads a host
band in one copy), so the factors, and the solution, agree bit for bit; a
pageable (unpinned) band takes the same path."""
import numpy as np
import pytest

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


CASES = [
    # n, k, p, r, precision, compress, reduced, nrhs
    (200011, 16, 40, 4, "fp32", "coupling", "truncated", 1),   # 16 groups of 2-3 partitions, side stream
    (150001, 64, 19, 16, "fp32", "coupling", "truncated", 3),  # KB = 64, ragged groups
    (60013, 32, 5, 8, "fp64", "spike", "full", 2),             # fewer partitions than groups, no side stream
    (50000, 8, 2, 2, "fp32", "spike", "truncated", 1),         # two partitions
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{}-k{}-p{}-{}-{}".format(c[0], c[1], c[2], c[4], c[5]))
@pytest.mark.parametrize("pinned", [True, False])
def test_host_band_equals_device_band(torch_cuda, case, pinned):
    torch = torch_cuda
    from paper_2504_11167_gb300.solver import LRSpike
    n, k, p, r, precision, compress, reduced, nrhs = case
    ab = inputs.dominant_band(n, k, 1.1, 300 + p)
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, nrhs, 300 + p).T)).cuda()
    hb = torch.from_numpy(ab)
    if pinned:
        hb = hb.pin_memory()
    db = hb.cuda()
    out = []
    # each handle factors twice (the second upload reuses its streams)
    for band, profile in ((db, False), (hb, True), (hb, False), (hb, False)):
        with LRSpike(n, k, p, r, precision=precision, compress=compress, reduced=reduced, tol=1e-10,
                     max_nrhs=nrhs, profile=profile) as s:
            s.factor(band)
            x, info = s.solve(f)
            assert info["converged"]
            s.factor(band)
            x2, _ = s.solve(f)
            out.append((x.clone(), x2.clone()))
    for x, x2 in out:
        assert torch.equal(x, out[0][0]) and torch.equal(x2, out[0][0])
