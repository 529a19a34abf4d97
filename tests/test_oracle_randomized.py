"""Pins of the oracle's randomized truncation (wide bands, k > 64).

The paper truncates the spikes with the randomized SVD of Halko, Martinsson
and Tropp (section 3.1): sketch the spike, orthonormalise, power passes, small
SVD of Q^T T.  What fixes the oracle here, independently of its own code: the
published output sequence of the SplitMix64 generator, the moments of the
Gaussian sketch, the special case ell = k (the randomized truncation must then
equal the exact truncated SVD, also for spectra spanning many orders of
magnitude), exactly low-rank inputs (recovered to rounding), the Eckart-Young
error of the exact truncation (the randomized one may not beat it and should
stay close to it on a fast-decaying spectrum, closer with power passes than
without), and wide-band solves (r = k reproduces A^{-1} to rounding).
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
    """ell = k: the basis spans range(X) and the truncation is the exact
    truncated SVD, up to rounding."""
    X, _ = decaying(600, 40, 1, rate=0.9)
    r = 6
    Ue, se, Ve, _ = O.truncated_svd(X, r, 1e-13)
    Ur, sr, Vr, _ = O.randomized_truncation(X, r, 40, 2, 99, 1e-13)
    assert np.allclose(sr, se, rtol=1e-12, atol=0)
    Te, Tr = (Ue * se) @ Ve, (Ur * sr) @ Vr
    assert np.linalg.norm(Tr - Te) <= 1e-12 * np.linalg.norm(Te)


def test_full_sketch_resolves_a_wide_spectrum():
    """Singular values from 1 down to 1e-12 (a Gram matrix X^T X would square
    them below FP64 resolution): with ell = r = k the sketch spans range(X) and
    X is reproduced to rounding, every singular value to ~eps relative to
    sigma_1."""
    X, s = decaying(500, 48, 4, rate=10 ** (-12 / 47))
    Ur, sr, Vr, _ = O.randomized_truncation(X, 48, 48, 2, 3, 1e-15)
    assert np.linalg.norm(X - (Ur * sr) @ Vr, 2) <= 1e-14 * s[0]
    assert np.all(np.abs(sr - s) <= 1e-14 * s[0])


def test_exactly_low_rank_input_is_recovered():
    """rank(X) = 7 <= r: Q spans range(X) whatever the sketch, so the
    truncation returns X itself (the rank <= r invariant of the survey)."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((400, 7)) @ rng.standard_normal((7, 90))
    for q in (0, 1, 2):
        Ur, sr, Vr, _ = O.randomized_truncation(X, 7, 12, q, 5, 1e-13)
        assert np.linalg.norm(X - (Ur * sr) @ Vr) <= 1e-13 * np.linalg.norm(X)


def test_power_passes_reduce_the_error():
    """Slowly decaying spectrum: each power pass raises the spectrum seen by
    the sketch to a higher power, so the error approaches sigma_{r+1}."""
    X, s = decaying(700, 120, 6, rate=0.97)
    r = 10
    errs = []
    for q in (0, 1, 3):
        Ur, sr, Vr, _ = O.randomized_truncation(X, r, 2 * r, q, 17, 1e-13)
        errs.append(np.linalg.norm(X - (Ur * sr) @ Vr, 2))
    assert errs[0] > errs[1] > errs[2] >= s[r] * (1 - 1e-9)
    assert errs[2] <= 1.1 * s[r]


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


def test_wide_band_full_rank_sketch_is_exact():
    """r = k, ell = k on a wide band: every truncated spike is the exact spike,
    so M^{-1} = A^{-1} (FULL reduced system) to rounding, and refinement needs
    one step; the exact truncated SVD gives the same."""
    n, k, p = 900, 70, 3
    ab = inputs.dominant_band(n, k, 1.5, 5)
    f = inputs.rhs(n, 1, 5)
    xs = np.linalg.solve(O.band_to_dense(ab, k), f)
    fac = O.factor(ab, k, p, k, reduced="full")
    assert np.linalg.norm(O.apply(fac, f) - xs) <= 1e-12 * np.linalg.norm(xs)
    assert O.ir_solve(ab, k, fac, f, tol=1e-12).iterations <= 1
    exact = O.factor(ab, k, p, k, reduced="full", randomized=False)
    assert np.linalg.norm(O.apply(exact, f) - xs) <= 1e-12 * np.linalg.norm(xs)
