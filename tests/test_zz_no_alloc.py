"""The allocation-free band residual, lrspike_residual_noalloc.

Some callers cannot allocate device memory: a serving loop in which a
cudaMalloc would synchronise the whole device and stall its other streams, or a
host framework that owns every device byte through its own pool.  For them the
library offers one entry point whose scratch is a static device array.  These
tests check its output against the existing entry point (lrspike_solve, which
reports the same quantity, ||f - A x|| / ||f|| per column, for its final
iterate) on two calls in a row, and that oversized or host arguments are
rejected.  The file is named so that pytest collects it last.
"""
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


def band_residual(torch, band, k, f, x):
    """f - A x with plain torch ops, one diagonal at a time."""
    n = band.shape[1]
    res = f.clone()
    for d in range(2 * k + 1):
        off = d - k                      # A[j + off, j] = band[d, j]
        lo, hi = max(0, -off), min(n, n - off)
        res[:, lo + off:hi + off] -= band[d, lo:hi] * x[:, lo:hi]
    return res


def test_noalloc_residual_matches_solve_entry_point(torch_cuda):
    torch = torch_cuda
    from paper_2504_11167_gb300.solver import LRSpike, residual_noalloc
    n, k, p, r, nrhs = 50021, 24, 6, 6, 3
    ab = inputs.dominant_band(n, k, 1.1, 31)
    band = torch.from_numpy(ab).cuda()
    f = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, nrhs, 31).T)).cuda()
    with LRSpike(n, k, p, r, precision="fp32", tol=1e-10) as s:
        s.factor(band)
        x, info = s.solve(f)
        x = x.clone()
    want = torch.tensor(info["rel_residual"], dtype=torch.float64)
    fnorm = torch.linalg.norm(f, dim=1)
    ref = band_residual(torch, band, k, f, x)
    scale = float((band.abs().sum(0).max() * x.abs().max()).item())
    for call in range(2):
        res = torch.full((nrhs, n), float("nan"), dtype=torch.float64, device="cuda")
        norms = torch.full((nrhs,), float("nan"), dtype=torch.float64, device="cuda")
        residual_noalloc(band, k, f, x, res, norms)
        torch.cuda.synchronize()
        got = (norms / fnorm).cpu()
        assert torch.allclose(got, want, rtol=1e-12, atol=0), (call, got, want)
        assert float((res - ref).abs().max()) <= 1e-12 * scale
        assert torch.allclose(torch.linalg.norm(res, dim=1), norms, rtol=1e-12, atol=0)


def test_noalloc_rejects_oversized_and_host_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2504_11167_gb300.solver import residual_noalloc
    n, k = 4096, 4
    band = torch.from_numpy(inputs.dominant_band(n, k, 1.5, 2)).cuda()
    f = torch.ones(1, n, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, n, dtype=torch.float64, device="cuda")
    res = torch.empty(1, n, dtype=torch.float64, device="cuda")
    norms = torch.empty(1, dtype=torch.float64, device="cuda")
    # the binding checks shapes and placement before it reaches the C call
    with pytest.raises(ValueError):
        residual_noalloc(band, k, f.cpu(), x, res, norms)
    with pytest.raises(ValueError):                 # x not the shape of f
        residual_noalloc(band, k, f, x[:, : n - 1], res, norms)
    with pytest.raises(ValueError):                 # r with a second column f does not have
        residual_noalloc(band, k, f, x, torch.empty(2, n, dtype=torch.float64, device="cuda"), norms)
    from paper_2504_11167_gb300.solver import load_library
    import ctypes
    lib = load_library()
    # the C entry point itself refuses host memory
    fh = f.cpu()
    st = lib.lrspike_residual_noalloc(ctypes.c_void_p(band.data_ptr()), n, n, k,
                                      ctypes.c_void_p(fh.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(res.data_ptr()), 1, n,
                                      ctypes.c_void_p(norms.data_ptr()), None)
    assert st == 1 and b"device memory" in lib.lrspike_last_error(None)
    # ceil(n / 256) * nrhs beyond the static scratch: refused before any GPU work
    big = 65536 * 256 + 1
    fake = torch.empty(1, 1, dtype=torch.float64, device="cuda")
    st = lib.lrspike_residual_noalloc(ctypes.c_void_p(band.data_ptr()), big, big, k,
                                      ctypes.c_void_p(fake.data_ptr()), ctypes.c_void_p(fake.data_ptr()),
                                      ctypes.c_void_p(fake.data_ptr()), 1, big,
                                      ctypes.c_void_p(fake.data_ptr()), None)
    assert st == 1 and b"static scratch" in lib.lrspike_last_error(None)
