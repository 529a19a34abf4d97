"""Pins of the oracle's randomized truncation (wide bands, k > 64).

The paper truncates the spikes with the randomized SVD of Halko, Martinsson
and Tropp (section 3.1).  What fixes the oracle here, independently of its own
code: the published output sequence of the SplitMix64 generator, the moments
of the Gaussian sketch, the special case ell = k (the randomized truncation
must then equal the exact truncated SVD), the Eckart-Young error of the exact
truncation (the randomized one may not beat it and should stay close to it on
a fast-decaying spectrum), and the final residual of a wide-band solve.
"""
import numpy as np
import pytest

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs


def test_splitmix64_published_sequence():
    # the reference implementation's outputs for seed 0 and seed 1234567
    assert [O.splitmix64(0, i) for i in range(4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [O.splitmix64(1234567, i) for i in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_gaussian_sketch_moments_and_reproducibility():
    om = O.gaussian_sketch(400, 50, 11)
    z = om.ravel()
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / z.size)
    assert abs(np.mean(z ** 4) - 3.0) < 0.3                     # normal kurtosis
    assert np.array_equal(om, O.gaussian_sketch(400, 50, 11))
    assert not np.array_equal(om[:, 0], O.gaussian_sketch(400, 50, 12)[:, 0])
    # entry (a, j) depends on the counter a*cols + j only
    assert O.gaussian_sketch(3, 4, 5)[2, 1] == O.gaussian_sketch(1, 12, 5)[0, 9]


def decaying(m, k, seed, rate=0.7):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = rate ** np.arange(k)
    return (U * s) @ V.T, s


def test_full_sketch_equals_exact_truncated_svd():
    """ell = k with every direction kept (sigma_k^2 / sigma_1^2 = 0.9^78 = 2.7e-4,
    far above the orthonormalisation cut of 1e-7): the basis spans R^k and the
    Rayleigh-Ritz step returns the exact truncated SVD, up to rounding."""
    X, _ = decaying(600, 40, 1, rate=0.9)
    r = 6
    Ue, se, Ve, _ = O.truncated_svd(X, r, 1e-13)
    Ur, sr, Vr, _ = O.randomized_truncation(X, r, 40, 2, 99, 1e-13)
    assert np.allclose(sr, se, rtol=1e-10, atol=0)
    Te, Tr = (Ue * se) @ Ve, (Ur * sr) @ Vr
    assert np.linalg.norm(Tr - Te) <= 1e-10 * np.linalg.norm(Te)


def test_randomized_error_close_to_eckart_young():
    X, s = decaying(800, 96, 2, rate=0.8)
    for r in (4, 8, 16):
        Ur, sr, Vr, _ = O.randomized_truncation(X, r, 2 * r, 2, 7 + r, 1e-13)
        err = np.linalg.norm(X - (Ur * sr) @ Vr, 2)
        assert err >= s[r] * (1 - 1e-9)          # no rank-r matrix beats sigma_{r+1}
        assert err <= 1.05 * s[r]                # oversampled, two passes: within 5 %


def test_rank_guard_drops_zero_directions():
    X, _ = decaying(300, 80, 3)
    X[:, 5:] = 0.0                                 # rank 5
    Ur, sr, Vr, _ = O.randomized_truncation(X, 8, 16, 2, 1, 1e-10)
    assert np.count_nonzero(sr) == 5
    assert np.linalg.norm(X - (Ur * sr) @ Vr) <= 1e-10 * np.linalg.norm(X)


def test_wide_band_factor_defaults_to_randomized_and_solves():
    n, k, p, r = 3000, 80, 4, 8
    ab = inputs.dominant_band(n, k, 1.3, 21)
    f = inputs.rhs(n, 1, 21)
    fac = O.factor(ab, k, p, r)                  # k > 64: randomized truncation
    res = O.ir_solve(ab, k, fac, f, tol=1e-12)
    assert res.converged
    exact = O.factor(ab, k, p, r, randomized=False)
    # same spikes, slightly different rank-r subspaces: the preconditioners agree closely
    g1, g2 = O.apply(fac, f), O.apply(exact, f)
    assert np.linalg.norm(g1 - g2) <= 1e-2 * np.linalg.norm(g2)


def test_wide_band_full_rank_sketch_is_near_exact_spike():
    """r = k, ell = k on a wide band: the exact truncation would give
    M^{-1} = A^{-1}; through G = T^T T the FP64 eigenvalues carry absolute
    errors ~ eps sigma_1^2, so spike directions below ~1e-4 sigma_1 (here the
    tail of a fast-decaying spike spectrum) are not resolved.  M^{-1} f then
    agrees with A^{-1} f to ~1e-5, each refinement step contracts the residual
    by ~1e-5, so 1e-12 takes at most three steps; the exact truncation stays
    exact to rounding."""
    n, k, p = 900, 70, 3
    ab = inputs.dominant_band(n, k, 1.5, 5)
    f = inputs.rhs(n, 1, 5)
    xs = np.linalg.solve(O.band_to_dense(ab, k), f)
    fac = O.factor(ab, k, p, k, reduced="full")
    assert np.linalg.norm(O.apply(fac, f) - xs) <= 1e-5 * np.linalg.norm(xs)
    assert O.ir_solve(ab, k, fac, f, tol=1e-12).iterations <= 3
    exact = O.factor(ab, k, p, k, reduced="full", randomized=False)
    assert np.linalg.norm(O.apply(exact, f) - xs) <= 1e-12 * np.linalg.norm(xs)
