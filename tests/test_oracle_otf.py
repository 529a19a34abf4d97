"""Pins of the oracle's LR-SPIKE-OTF (section 2.2 "SPIKE-on-the-fly", eqs.
OTF-1/OTF-2; section 3.3, the truncated low-rank reduced system as its
preconditioner) against quantities computed independently of it:

* the on-the-fly reduced operator equals the reduced operator assembled from
  explicit spikes V_i = A_i^{-1}[0; B_i], W_i = A_i^{-1}[C_i; 0] formed with
  dense solves (numpy.linalg.solve on the dense A_i, not the oracle's band LU);
* with r = k (no truncation) the Woodbury preconditioner inverts the explicit
  per-interface block [[I, V_{i,b}], [W_{i+1,t}, I]];
* one OTF solve with a tight reduced tolerance reproduces x = A^{-1} f from
  LAPACK's banded solver, and the refinement around it reaches the tolerance.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs


def dense_spikes(ab, k, offs):
    """Explicit tips of V_i and W_i from dense solves: returns per partition
    (V_top, V_bot, W_top, W_bot), each k x k (None where the spike is absent)."""
    A = O.band_to_dense(ab, k)
    p = len(offs) - 1
    out = []
    for i in range(p):
        s, e = int(offs[i]), int(offs[i + 1])
        Ai = A[s:e, s:e]
        VT = VB = WT = WB = None
        if i < p - 1:  # V_i = A_i^{-1} [0; B_i], B_i = A[e-k:e, e:e+k]
            rhs = np.zeros((e - s, k))
            rhs[-k:] = A[e - k:e, e:e + k]
            V = np.linalg.solve(Ai, rhs)
            VT, VB = V[:k], V[-k:]
        if i > 0:  # W_i = A_i^{-1} [C_i; 0], C_i = A[s:s+k, s-k:s]
            rhs = np.zeros((e - s, k))
            rhs[:k] = A[s:s + k, s - k:s]
            W = np.linalg.solve(Ai, rhs)
            WT, WB = W[:k], W[-k:]
        out.append((VT, VB, WT, WB))
    return out


def explicit_S(sp, k, p, y):
    """The reduced operator from explicit spike tips (unknowns per interface
    i: [x_{i,b}; x_{i+1,t}])."""
    out = y.copy()
    for i in range(p - 1):
        xb, xt = y[i, :k], y[i, k:]
        # bottom tip of partition i: + V_{i,b} x_{i+1,t} + W_{i,b} x_{i-1,b}
        out[i, :k] += sp[i][1] @ xt
        if i > 0:
            out[i, :k] += sp[i][3] @ y[i - 1, :k]
        # top tip of partition i+1: + W_{i+1,t} x_{i,b} + V_{i+1,t} x_{i+2,t}
        out[i, k:] += sp[i + 1][2] @ xb
        if i + 1 < p - 1:
            out[i, k:] += sp[i + 1][0] @ y[i + 1, k:]
    return out


CASES = [(600, 6, 4, 3), (900, 10, 5, 4), (700, 12, 3, 12)]


@pytest.mark.parametrize("n,k,p,r", CASES)
def test_otf_operator_equals_explicit_spikes(n, k, p, r):
    ab = inputs.dominant_band(n, k, 1.3, 60 + n)
    fac = O.factor(ab, k, p, r, reduced="truncated")
    sp = dense_spikes(ab, k, fac.offs)
    rng = np.random.default_rng(3)
    y = rng.standard_normal((p - 1, 2 * k, 2))
    got = O.otf_S(fac, ab, y)
    for q in range(2):
        ref = explicit_S(sp, k, p, y[:, :, q])
        assert np.abs(got[:, :, q] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_otf_preconditioner_inverts_the_interface_block_at_full_rank():
    n, k, p = 800, 8, 4
    r = k  # exact spikes: T~ = T, W~ = W
    ab = inputs.dominant_band(n, k, 1.2, 71)
    fac = O.factor(ab, k, p, r, reduced="truncated")
    sp = dense_spikes(ab, k, fac.offs)
    rng = np.random.default_rng(5)
    y = rng.standard_normal((p - 1, 2 * k, 1))
    # the truncated interface blocks applied explicitly
    My = y.copy()
    for i in range(p - 1):
        My[i, :k, 0] += sp[i][1] @ y[i, k:, 0]       # V_{i,b} x_{i+1,t}
        My[i, k:, 0] += sp[i + 1][2] @ y[i, :k, 0]   # W_{i+1,t} x_{i,b}
    back = O.otf_prec(fac, My)
    assert np.abs(back - y).max() <= 1e-10 * np.abs(y).max()


@pytest.mark.parametrize("compress", ["spike", "coupling"])
def test_otf_solve_reproduces_the_banded_solution(compress):
    n, k, p, r = 3000, 8, 6, 3
    ab = inputs.dominant_band(n, k, 1.2, 81)
    f = inputs.rhs(n, 2, 81)
    fac = O.factor(ab, k, p, r, compress=compress, reduced="truncated")
    x, its = O.otf_apply(fac, ab, f, otf_tol=1e-13, max_iter=200)
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert 1 <= its < 60
    # a looser reduced tolerance leaves an error of about that size, which
    # refinement around the OTF solve removes
    res = O.otf_solve(ab, k, fac, f, tol=1e-12, otf_tol=1e-6)
    assert res.converged and res.iterations <= 4


def test_otf_beats_the_truncated_preconditioner_alone():
    """The true reduced system: one OTF solve is far closer to A^{-1} f than
    one application of the truncated low-rank preconditioner it uses."""
    n, k, p, r = 2000, 8, 8, 2
    ab = inputs.dominant_band(n, k, 1.05, 91)
    f = inputs.rhs(n, 1, 91)
    fac = O.factor(ab, k, p, r, reduced="truncated")
    xs = scipy.linalg.solve_banded((k, k), ab, f)
    x_otf, _ = O.otf_apply(fac, ab, f, otf_tol=1e-10)
    x_pre = O.apply(fac, f)
    e_otf = np.linalg.norm(x_otf - xs) / np.linalg.norm(xs)
    e_pre = np.linalg.norm(x_pre - xs) / np.linalg.norm(xs)
    assert e_otf <= 1e-8 and e_otf < 1e-3 * e_pre
