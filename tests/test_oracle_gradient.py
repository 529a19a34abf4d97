"""Pin of the oracle's solve gradient (the adjoint of x = A^{-1} f) by
central differences of L = 0.5 |x - x*|^2 with dense solves on a tiny band:
dL/df = lambda = A^{-T}(x - x*) and dL/dA_ij = -lambda_i x_j on the band."""
import numpy as np

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs


def loss(ab, k, f, xs):
    x = np.linalg.solve(O.band_to_dense(ab, k), f)
    return 0.5 * np.sum((x - xs) ** 2)


def test_gradient_matches_central_differences():
    n, k = 30, 3
    ab = inputs.dominant_band(n, k, 1.4, 3)
    f = inputs.rhs(n, 1, 3)[:, 0]
    xs = inputs.target(n, 1, 3)[:, 0]
    x, lam, G = O.solve_gradients(ab, k, f, lambda x: x - xs)
    h = 1e-5
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        fd = (loss(ab, k, f + e, xs) - loss(ab, k, f - e, xs)) / (2 * h)
        assert abs(fd - lam[j]) <= 1e-7 * (1 + abs(lam[j]))
    for d in range(2 * k + 1):
        for j in range(n):
            i = j + d - k
            if not 0 <= i < n:
                assert G[d, j] == 0.0
                continue
            a1, a2 = ab.copy(), ab.copy()
            a1[d, j] += h
            a2[d, j] -= h
            fd = (loss(a1, k, f, xs) - loss(a2, k, f, xs)) / (2 * h)
            assert abs(fd - G[d, j]) <= 1e-7 * (1 + abs(G[d, j]))
