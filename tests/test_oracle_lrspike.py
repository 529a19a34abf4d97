"""Pins for the LR-SPIKE oracle.  Each pin is fixed by the paper or by mathematics,
not by re-running the oracle's own formula:

* r = k with the FULL reduced system is exact SPIKE, so M^{-1} f = A^{-1} f
  (dense LU brute force);  p = 1 gives the plain band solve;
* r = 0 is Block Jacobi (section 4.1: the limiting case n_svd = 0);
* FULL with r < k equals (D S~)^{-1} f with S~ built densely from the
  low-rank spikes (section 3.2: S~ is S with the spikes replaced by T~, W~);
* TRUNCATED equals the paper's own per-interface form: 2k x 2k blocks
  [[I, T~_{i,b}], [W~_{i+1,t}, I]] inverted through the Schur complement M_i and
  the Woodbury identity (section 3.2, eqs. 'red_sys_mid', 'red_sys_prec_inv'),
  followed by low-rank recovery; at p = 2 TRUNCATED equals FULL (the 2x2 kernel);
* the compression obeys Eckart-Young, ||T - T~||_2 = sigma_{r+1} (section 3.1),
  checked with a symmetric eigensolver instead of an SVD;
* couplings of rank <= r are reproduced exactly by either compression mode;
* the transposed operator equals the transpose of the dense M^{-1};
* IR and BiCGStab reach the requested residual.
A last group plants plausible mistakes in the oracle and checks that the pins
catch them.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs


def make(n, k, dom=1.5, seed=1):
    return inputs.dominant_band(n, k, dom, seed)


def dense_solve(ab, k, f):
    return np.linalg.solve(O.band_to_dense(ab, k), f)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def explicit_spikes(ab, k, fac):
    """Dense T_i = A_i^{-1}[0; B_i] and W_i = A_i^{-1}[C_i; 0] by numpy solves."""
    A = O.band_to_dense(ab, k)
    T, W = [], []
    for i in range(fac.p):
        s, e = int(fac.offs[i]), int(fac.offs[i + 1])
        Ai = A[s:e, s:e]
        if i < fac.p - 1:
            rhs = np.zeros((e - s, k))
            rhs[-k:] = A[e - k:e, e:e + k]
            T.append(np.linalg.solve(Ai, rhs))
        else:
            T.append(None)
        if i > 0:
            rhs = np.zeros((e - s, k))
            rhs[:k] = A[s:s + k, s - k:s]
            W.append(np.linalg.solve(Ai, rhs))
        else:
            W.append(None)
    return T, W


def test_partition_offsets():
    offs = O.partition_offsets(103, 4)
    assert list(np.diff(offs)) == [26, 26, 26, 25] and offs[-1] == 103
    assert list(O.partition_offsets(64, 8)) == list(range(0, 65, 8))


def test_coupling_blocks_are_dense_slices():
    n, k, p = 90, 5, 3
    ab = make(n, k)
    A = O.band_to_dense(ab, k)
    offs = O.partition_offsets(n, p)
    for i in range(p - 1):
        s = int(offs[i + 1])
        B = O.coupling_B(ab, k, s)
        C = O.coupling_C(ab, k, s)
        assert np.array_equal(B, A[s - k:s, s:s + k]) and np.allclose(np.triu(B, 1), 0)
        assert np.array_equal(C, A[s:s + k, s - k:s]) and np.allclose(np.tril(C, -1), 0)


def test_spike_definition():
    n, k, p = 120, 6, 3
    ab = make(n, k, seed=4)
    fac = O.factor(ab, k, p, r=k)
    T, W = explicit_spikes(ab, k, fac)
    A = O.band_to_dense(ab, k)
    for i in range(p):
        s, e = int(fac.offs[i]), int(fac.offs[i + 1])
        if i < p - 1:
            lhs = A[s:e, s:e] @ (fac.UV[i] @ fac.PV[i])
            rhs = np.zeros((e - s, k))
            rhs[-k:] = A[e - k:e, e:e + k]
            assert np.abs(lhs - rhs).max() < 1e-12
        if i > 0:
            lhs = A[s:e, s:e] @ (fac.UW[i] @ fac.QW[i])
            rhs = np.zeros((e - s, k))
            rhs[:k] = A[s:s + k, s - k:s]
            assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("compress", ["spike", "coupling"])
@pytest.mark.parametrize("n,k,p", [(200, 8, 4), (131, 5, 3), (400, 16, 5)])
def test_full_rank_full_reduced_is_exact(n, k, p, compress):
    ab = make(n, k, seed=n + k)
    f = inputs.rhs(n, 2, seed=7)
    fac = O.factor(ab, k, p, r=k, compress=compress, reduced="full")
    assert rel(O.apply(fac, f), dense_solve(ab, k, f)) < 1e-12


def test_single_partition_is_band_solve():
    n, k = 150, 7
    ab = make(n, k, dom=1.1, seed=3)
    f = inputs.rhs(n, 1, seed=3)
    fac = O.factor(ab, k, 1, r=3)
    x = O.apply(fac, f)
    assert rel(x, scipy.linalg.solve_banded((k, k), ab, f)) < 1e-13


def test_rank_zero_is_block_jacobi():
    n, k, p = 180, 6, 3
    ab = make(n, k, seed=8)
    f = inputs.rhs(n, 1, seed=8)
    fac = O.factor(ab, k, p, r=0)
    A = O.band_to_dense(ab, k)
    D = np.zeros_like(A)
    for i in range(p):
        s, e = int(fac.offs[i]), int(fac.offs[i + 1])
        D[s:e, s:e] = A[s:e, s:e]
    assert rel(O.apply(fac, f), np.linalg.solve(D, f)) < 1e-13


def dense_S_tilde(fac):
    """I plus the low-rank spikes T~_i = u P_i (columns of x_{i+1,t}) and
    W~_i = u Q_i (columns of x_{i-1,b}), eq. 'DS_first' with T, W replaced."""
    n, k = fac.n, fac.k
    S = np.eye(n)
    for i in range(fac.p):
        s, e = int(fac.offs[i]), int(fac.offs[i + 1])
        if i < fac.p - 1:
            S[s:e, e:e + k] += fac.UV[i] @ fac.PV[i]
        if i > 0:
            S[s:e, s - k:s] += fac.UW[i] @ fac.QW[i]
    return S


@pytest.mark.parametrize("compress", ["spike", "coupling"])
@pytest.mark.parametrize("n,k,p,r", [(240, 8, 4, 3), (150, 6, 3, 1), (333, 12, 5, 5)])
def test_full_low_rank_equals_dense_DS(n, k, p, r, compress):
    ab = make(n, k, dom=1.1, seed=2 * n + r)
    f = inputs.rhs(n, 2, seed=1)
    fac = O.factor(ab, k, p, r=r, compress=compress, reduced="full")
    A = O.band_to_dense(ab, k)
    D = np.zeros_like(A)
    for i in range(p):
        s, e = int(fac.offs[i]), int(fac.offs[i + 1])
        D[s:e, s:e] = A[s:e, s:e]
    M = D @ dense_S_tilde(fac)
    assert rel(O.apply(fac, f), np.linalg.solve(M, f)) < 1e-12


def paper_truncated_apply(ab, k, fac, f):
    """The paper's LR-SPIKE-T solve in x-tip space, independent of the oracle's
    compressed reduced system: D-stage by dense solves, then for every
    interface the block inverse of [[I, T~_{i,b}], [W~_{i+1,t}, I]] through
    M_i = I - W~_{i+1,t} T~_{i,b} with M_i^{-1} from the Woodbury form
    (eq. 'red_sys_prec_inv'), then recovery with the low-rank spikes."""
    A = O.band_to_dense(ab, k)
    p, offs = fac.p, fac.offs
    g = np.zeros_like(f)
    for i in range(p):
        s, e = int(offs[i]), int(offs[i + 1])
        g[s:e] = np.linalg.solve(A[s:e, s:e], f[s:e])
    xb, xt = {}, {}
    for i in range(p - 1):
        e = int(offs[i + 1])
        uVb, SvV = fac.UV[i][-k:], fac.PV[i]            # T~_{i,b} = u_{T,b} (Sigma v)_T
        uWt, SvW = fac.UW[i + 1][:k], fac.QW[i + 1]     # W~_{i+1,t} = u_{W,t} (Sigma v)_W
        sigW = np.linalg.norm(SvW, axis=1)
        vW = SvW / sigW[:, None]
        C = vW @ uVb                                    # v_W u_{T,b}  (n_svd x n_svd)
        inner = np.linalg.inv(C) - SvV @ uWt @ np.diag(sigW)
        Minv = np.eye(k) + uWt @ np.diag(sigW) @ np.linalg.solve(inner, SvV)
        Tb = uVb @ SvV
        Wt = uWt @ SvW
        gb, gt = g[e - k:e], g[e:e + k]
        xb[i] = (gb + Tb @ Minv @ Wt @ gb) - Tb @ Minv @ gt
        xt[i + 1] = -Minv @ Wt @ gb + Minv @ gt
    x = g.copy()
    for i in range(p):
        s, e = int(offs[i]), int(offs[i + 1])
        if i < p - 1:
            x[s:e] -= fac.UV[i] @ fac.PV[i] @ xt[i + 1]
        if i > 0:
            x[s:e] -= fac.UW[i] @ fac.QW[i] @ xb[i - 1]
    return x


@pytest.mark.parametrize("n,k,p,r", [(320, 8, 4, 3), (500, 10, 5, 4), (240, 6, 3, 6)])
def test_truncated_equals_paper_woodbury_form(n, k, p, r):
    ab = make(n, k, dom=1.05, seed=n)
    f = inputs.rhs(n, 1, seed=2)
    fac = O.factor(ab, k, p, r=r, compress="spike", reduced="truncated")
    assert rel(O.apply(fac, f), paper_truncated_apply(ab, k, fac, f)) < 1e-11


def test_two_partitions_truncated_equals_full():
    n, k = 160, 8
    ab = make(n, k, dom=1.05, seed=5)
    f = inputs.rhs(n, 1, seed=5)
    a = O.apply(O.factor(ab, k, 2, r=3, reduced="truncated"), f)
    b = O.apply(O.factor(ab, k, 2, r=3, reduced="full"), f)
    assert rel(a, b) < 1e-14


def _two_norm(X):
    return np.sqrt(max(np.linalg.eigvalsh(X.T @ X).max(), 0.0))


def test_eckart_young_for_spikes_and_couplings():
    n, k, p, r = 300, 10, 3, 4
    ab = make(n, k, dom=1.2, seed=9)
    fac = O.factor(ab, k, p, r=r, compress="spike")
    T, W = explicit_spikes(ab, k, fac)
    for i in range(p - 1):
        lam = np.sort(np.linalg.eigvalsh(T[i].T @ T[i]))[::-1]
        err = _two_norm(T[i] - fac.UV[i] @ fac.PV[i])
        assert abs(err - np.sqrt(lam[r])) < 1e-9 * np.sqrt(lam[0])
    for i in range(1, p):
        lam = np.sort(np.linalg.eigvalsh(W[i].T @ W[i]))[::-1]
        err = _two_norm(W[i] - fac.UW[i] @ fac.QW[i])
        assert abs(err - np.sqrt(lam[r])) < 1e-9 * np.sqrt(lam[0])
    # COUPLING: T~ = A_i^{-1}[0; B_r] with B_r the best rank-r approximation of B_i
    fc = O.factor(ab, k, p, r=r, compress="coupling")
    A = O.band_to_dense(ab, k)
    for i in range(p - 1):
        s, e = int(fc.offs[i]), int(fc.offs[i + 1])
        B = A[e - k:e, e:e + k]
        Br = (A[s:e, s:e] @ (fc.UV[i] @ fc.PV[i]))[-k:]
        lam = np.sort(np.linalg.eigvalsh(B.T @ B))[::-1]
        assert abs(_two_norm(B - Br) - np.sqrt(lam[r])) < 1e-9 * np.sqrt(lam[0])
        assert np.abs((A[s:e, s:e] @ (fc.UV[i] @ fc.PV[i]))[:-k]).max() < 1e-12


@pytest.mark.parametrize("compress", ["spike", "coupling"])
def test_low_rank_couplings_are_exact(compress):
    n, k, p, r = 400, 8, 4, 3
    offs = O.partition_offsets(n, p)
    ab = inputs.low_rank_coupling_band(n, k, p, r, 1.3, 21, offs)
    A = O.band_to_dense(ab, k)
    for i in range(p - 1):
        s = int(offs[i + 1])
        assert np.linalg.matrix_rank(A[s - k:s, s:s + k]) <= r
        assert np.linalg.matrix_rank(A[s:s + k, s - k:s]) <= r
    f = inputs.rhs(n, 1, seed=4)
    fac = O.factor(ab, k, p, r=r, compress=compress, reduced="full")
    assert rel(O.apply(fac, f), np.linalg.solve(A, f)) < 1e-11


def dense_precond(fac):
    return O.apply(fac, np.eye(fac.n))


@pytest.mark.parametrize("reduced", ["full", "truncated"])
@pytest.mark.parametrize("pivoting", [False, True])
def test_transpose_is_dense_transpose(reduced, pivoting):
    n, k, p, r = 96, 4, 3, 2
    ab = make(n, k, dom=0.3 if pivoting else 1.2, seed=13)
    fac = O.factor(ab, k, p, r=r, reduced=reduced, pivoting=pivoting)
    if pivoting:
        assert any(np.any(pt.ipiv != np.arange(pt.n)) for pt in fac.parts)
    Minv = dense_precond(fac)
    h = inputs.rhs(n, 2, seed=6)
    assert rel(O.apply_T(fac, h), Minv.T @ h) < 1e-12
    # adjoint identity <M^{-1} f, g> = <f, M^{-T} g>
    f, g = h[:, 0], h[:, 1]
    a, b = O.apply(fac, f) @ g, f @ O.apply_T(fac, g)
    assert abs(a - b) < 1e-13 * max(abs(a), 1.0)


def test_pivoted_partitions_exact_at_full_rank():
    n, k, p = 240, 6, 3
    ab = make(n, k, dom=0.05, seed=17)
    f = inputs.rhs(n, 1, seed=17)
    fac = O.factor(ab, k, p, r=k, pivoting=True)
    assert any(np.any(pt.ipiv != np.arange(pt.n)) for pt in fac.parts)
    assert rel(O.apply(fac, f), dense_solve(ab, k, f)) < 1e-10


@pytest.mark.parametrize("reduced", ["full", "truncated"])
def test_ir_reaches_tolerance(reduced):
    n, k, p, r = 8192, 16, 8, 4
    ab = make(n, k, dom=1.5, seed=inputs.SEED_BASE + 1)
    f = inputs.rhs(n, 1, seed=inputs.SEED_BASE + 1)
    fac = O.factor(ab, k, p, r=r, reduced=reduced)
    res = O.ir_solve(ab, k, fac, f, tol=1e-12)
    assert res.converged and res.rel_residual.max() <= 1e-12
    x = scipy.linalg.solve_banded((k, k), ab, f)
    assert rel(res.x, x) < 1e-10
    rt = O.ir_solve(ab, k, fac, f, tol=1e-12, trans=True)
    A_T_solution = scipy.linalg.solve_banded((k, k), O_band_transpose(ab, k), f)
    assert rt.converged and rel(rt.x, A_T_solution) < 1e-10


def O_band_transpose(ab, k):
    """Band of A^T: A^T[i, j] = A[j, i] -> row k+i-j of column j holds A[j, i]."""
    n = ab.shape[1]
    at = np.zeros_like(ab)
    for d in range(2 * k + 1):
        off = d - k              # A[j+off, j] = ab[d, j]  ->  A^T[j, j+off]
        for j in range(n):
            i = j + off
            if 0 <= i < n:
                at[k + j - i, i] = ab[d, j]
    return at


def test_bicgstab_reaches_tolerance():
    n, k, p, r = 2000, 8, 5, 2
    ab = make(n, k, dom=1.02, seed=31)
    f = inputs.rhs(n, 2, seed=31)
    fac = O.factor(ab, k, p, r=r, reduced="truncated")
    res = O.bicgstab(ab, k, fac, f, tol=1e-12)
    assert res.converged
    assert rel(res.x, dense_solve(ab, k, f)) < 1e-9


def test_quality_improves_with_rank_and_spike_beats_coupling():
    n, k, p = 240, 8, 4
    ab = make(n, k, dom=1.01, seed=41)
    A = O.band_to_dense(ab, k)
    errs = {}
    for r in (0, 2, 4, 8):
        for compress in ("spike", "coupling"):
            Minv = dense_precond(O.factor(ab, k, p, r=r, compress=compress))
            errs[r, compress] = np.linalg.norm(np.eye(n) - Minv @ A, 2)
    assert errs[0, "spike"] > errs[2, "spike"] > errs[4, "spike"] > errs[8, "spike"]
    assert errs[8, "spike"] < 1e-12
    for r in (2, 4):
        assert errs[r, "spike"] <= errs[r, "coupling"] + 1e-12


# ---------------------------------------------------------------------------
# Planted mistakes: each plausible slip in the oracle must break a pin above.
# ---------------------------------------------------------------------------
def _exactness_error(ab, k, p, f):
    fac = O.factor(ab, k, p, r=k, reduced="full")
    return rel(O.apply(fac, f), dense_solve(ab, k, f))


def test_planted_mistakes_are_caught(monkeypatch):
    n, k, p = 200, 8, 4
    ab = make(n, k, seed=77)
    f = inputs.rhs(n, 1, seed=77)
    assert _exactness_error(ab, k, p, f) < 1e-12

    orig_V = O.V_op

    def V_swapped(fac, x):              # uses the bottom tip where the top tip belongs
        k_, r, offs = fac.k, fac.r, fac.offs
        X = x.reshape(fac.n, -1)
        z = np.zeros((fac.nz, X.shape[1]))
        for i in range(fac.p - 1):
            s = int(offs[i + 1])
            z[2 * r * i: 2 * r * i + r] = fac.PV[i] @ X[s - k_: s]
            z[2 * r * i + r: 2 * r * (i + 1)] = fac.QW[i + 1] @ X[s: s + k_]
        return z
    monkeypatch.setattr(O, "V_op", V_swapped)
    assert _exactness_error(ab, k, p, f) > 1e-6
    monkeypatch.setattr(O, "V_op", orig_V)

    orig_U = O.U_op

    def U_shifted(fac, z):              # omega_i read from interface i instead of i-1
        r, offs = fac.r, fac.offs
        Z = z.reshape(fac.nz, -1)
        x = np.zeros((fac.n, Z.shape[1]))
        for i in range(fac.p):
            s, e = int(offs[i]), int(offs[i + 1])
            if i < fac.p - 1:
                x[s:e] += fac.UV[i] @ Z[2 * r * i: 2 * r * i + r]
                if i > 0:
                    x[s:e] += fac.UW[i] @ Z[2 * r * i + r: 2 * r * (i + 1)]
        return x
    monkeypatch.setattr(O, "U_op", U_shifted)
    assert _exactness_error(ab, k, p, f) > 1e-6
    monkeypatch.setattr(O, "U_op", orig_U)

    orig_B = O.coupling_B
    monkeypatch.setattr(O, "coupling_B", lambda ab_, k_, s: orig_B(ab_, k_, s).T)
    assert _exactness_error(ab, k, p, f) > 1e-6
    monkeypatch.setattr(O, "coupling_B", orig_B)

    orig_apply = O.apply

    def apply_sign(fac, f_):             # recovery with + instead of -
        g = O.d_solve(fac, f_)
        z = scipy.linalg.lu_solve(fac.R_lu, O.V_op(fac, g))
        return (g.reshape(fac.n, -1) + O.U_op(fac, z)).reshape(f_.shape)
    monkeypatch.setattr(O, "apply", apply_sign)
    assert _exactness_error(ab, k, p, f) > 1e-6
    monkeypatch.setattr(O, "apply", orig_apply)

    orig_trunc = O.truncate_R
    monkeypatch.setattr(O, "truncate_R", lambda R, r, p_: np.eye(R.shape[0]))
    fac = O.factor(ab, k, p, r=3, reduced="truncated")
    assert rel(O.apply(fac, f), paper_truncated_apply(ab, k, fac, f)) > 1e-8
    monkeypatch.setattr(O, "truncate_R", orig_trunc)
