"""Differentiable solve (torch.autograd.Function over the C ABI): backward =
adjoint solve with the stored factors (lrspike_solve_transpose) and the
band-restricted outer product (lrspike_band_outer).

Checks: central finite differences (step 1e-6) of L = 0.5 |x - x*|^2 on an
n = 4096, k = 32, p = 8, r = 8 FP64 instance for 64 band entries and 16
entries of f, and the oracle's exact gradient (LAPACK banded solves) to 1e-8.
Tolerances: L itself is O(n) here (x* is uniform[-1, 1]), so rounding L to a
few ulps puts ~10 eps |L| / h of absolute noise into each central-difference
quotient (~1.5e-6 at |L| = 700, h = 1e-6); the solves run to 1e-14, well below
that.  The FD bound is that noise plus 1e-6 of the gradient's scale (the
O(h^2) truncation is far smaller).
"""
import numpy as np
import pytest

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


N, K, P, R = 4096, 32, 8, 8


def setup(torch):
    ab = inputs.dominant_band(N, K, 1.5, 41)
    f = inputs.rhs(N, 1, 41)[:, 0]
    xs = inputs.target(N, 1, 41)[:, 0]
    return ab, f, xs


def loss_and_grads(torch, ab, f, xs, tol=1e-14):
    from paper_2504_11167_gb300.autograd import solve
    band = torch.from_numpy(ab).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    x = solve(band, ft, K, P, R, tol=tol, max_iter=100)
    loss = 0.5 * ((x - torch.from_numpy(xs).cuda()) ** 2).sum()
    loss.backward()
    return float(loss.detach()), band.grad.cpu().numpy(), ft.grad.cpu().numpy(), x.detach().cpu().numpy()


def test_gradient_matches_oracle(torch_cuda):
    torch = torch_cuda
    ab, f, xs = setup(torch)
    _, gA, gf, x = loss_and_grads(torch, ab, f, xs)
    xo, lam, G = O.solve_gradients(ab, K, f, lambda v: v - xs)
    assert np.linalg.norm(x - xo) <= 1e-12 * np.linalg.norm(xo)
    assert np.linalg.norm(gf - lam) <= 1e-8 * np.linalg.norm(lam)
    assert np.linalg.norm(gA - G) <= 1e-8 * np.linalg.norm(G)


def test_gradient_matches_central_differences(torch_cuda):
    torch = torch_cuda
    from paper_2504_11167_gb300.autograd import solve
    ab, f, xs = setup(torch)
    L0, gA, gf, _ = loss_and_grads(torch, ab, f, xs)
    rng = np.random.default_rng(5)
    h = 1e-6
    noise = 10 * np.finfo(float).eps * abs(L0) / h

    def L(a, g):
        with torch.no_grad():
            x = solve(torch.from_numpy(a).cuda(), torch.from_numpy(g).cuda(), K, P, R, tol=1e-14, max_iter=100)
            return 0.5 * float(((x - torch.from_numpy(xs).cuda()) ** 2).sum())

    scale_f = np.abs(gf).max()
    for j in rng.choice(N, 16, replace=False):
        e = np.zeros(N)
        e[j] = h
        fd = (L(ab, f + e) - L(ab, f - e)) / (2 * h)
        assert abs(fd - gf[j]) <= noise + 1e-6 * scale_f
    scale_A = np.abs(gA).max()
    picked = 0
    while picked < 64:
        d, j = int(rng.integers(0, 2 * K + 1)), int(rng.integers(0, N))
        if not 0 <= j + d - K < N:
            continue
        a1, a2 = ab.copy(), ab.copy()
        a1[d, j] += h
        a2[d, j] -= h
        fd = (L(a1, f) - L(a2, f)) / (2 * h)
        assert abs(fd - gA[d, j]) <= noise + 1e-6 * scale_A, (d, j, fd, gA[d, j])
        picked += 1


def test_mixed_precision_gradient(torch_cuda):
    """FP32 factors with FP64 refinement on both the solve and the adjoint:
    the gradient still matches the oracle to the refinement tolerance."""
    torch = torch_cuda
    from paper_2504_11167_gb300.autograd import solve
    ab, f, xs = setup(torch)
    band = torch.from_numpy(ab).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    x = solve(band, ft, K, P, R, precision="fp32", tol=1e-12, max_iter=100)
    (0.5 * ((x - torch.from_numpy(xs).cuda()) ** 2).sum()).backward()
    _, lam, G = O.solve_gradients(ab, K, f, lambda v: v - xs)
    assert np.linalg.norm(ft.grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)
    assert np.linalg.norm(band.grad.cpu().numpy() - G) <= 1e-9 * np.linalg.norm(G)
