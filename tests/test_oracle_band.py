"""Pins for the oracle's plain-C band routines against independent references:
numpy dense LU solves, LAPACK's dgbtrf / dgbtrs / gbsv (through scipy) and the
reconstruction L U = A of the factors."""
import numpy as np
import pytest
import scipy.linalg
from scipy.linalg import lapack

from oracle import lrspike_oracle as O
from paper_2504_11167_gb300 import inputs


def _dense_L_U_nopiv(lu: O.BandLU):
    n, k = lu.n, lu.k
    L, U = np.eye(n), np.zeros((n, n))
    st = lu.store
    for d in range(2 * k + 1):
        for j in range(n):
            i = j + d - k
            if 0 <= i < n:
                (U if i <= j else L)[i, j] = st[d, j]
    return L, U


@pytest.mark.parametrize("n,k", [(1, 0), (7, 1), (40, 3), (65, 8), (33, 32), (200, 16)])
def test_lu_nopiv_reconstructs_A(n, k):
    ab = inputs.dominant_band(n, k, 1.5, seed=3 + n + k)
    if n == 1:
        ab[k, 0] = 2.0
    lu = O.BandLU(ab, k, pivoting=False)
    L, U = _dense_L_U_nopiv(lu)
    A = O.band_to_dense(ab, k)
    assert np.allclose(L @ U, A, rtol=0, atol=1e-13 * np.abs(A).max())
    assert np.allclose(np.tril(U, -1), 0) and np.allclose(np.triu(U, k + 1), 0)


@pytest.mark.parametrize("n,k,nrhs", [(50, 4, 1), (129, 16, 3), (300, 7, 2)])
def test_solves_match_dense_and_lapack(n, k, nrhs):
    ab = inputs.dominant_band(n, k, 1.2, seed=11 + k)
    A = O.band_to_dense(ab, k)
    f = inputs.rhs(n, nrhs, seed=5)
    lu = O.BandLU(ab, k, pivoting=False)
    x = lu.solve(f)
    xd = np.linalg.solve(A, f)
    xs = scipy.linalg.solve_banded((k, k), ab, f)          # LAPACK gbsv
    assert np.linalg.norm(x - xd) <= 1e-13 * np.linalg.norm(xd)
    assert np.linalg.norm(x - xs) <= 1e-13 * np.linalg.norm(xs)
    xt = lu.solve(f, trans=True)
    assert np.linalg.norm(xt - np.linalg.solve(A.T, f)) <= 1e-13 * np.linalg.norm(xt)
    # matvec against the dense product, both orientations
    y = np.asarray(f)
    assert np.allclose(O.band_matvec(ab, k, y), A @ y, rtol=0, atol=1e-12)
    assert np.allclose(O.band_matvec(ab, k, y, trans=True), A.T @ y, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,k", [(60, 3), (150, 8), (257, 16), (96, 31)])
def test_pivoted_lu_matches_lapack_gbtrf(n, k):
    # a weak diagonal (0.05 x row sum) so that partial pivoting actually swaps rows;
    # at 0.6 a random band rarely needs a swap (its diagonal still beats every entry)
    ab = inputs.dominant_band(n, k, 0.05, seed=100 + n)
    lu = O.BandLU(ab, k, pivoting=True)
    lapack_ab = np.zeros((3 * k + 1, n))
    lapack_ab[k:, :] = ab
    lub, ipiv, info = lapack.dgbtrf(lapack_ab, k, k)
    assert info == 0
    # k < 32 keeps dgbtrf on its unblocked path: identical pivot sequence
    assert np.array_equal(lu.ipiv, ipiv.astype(np.int32))
    assert np.count_nonzero(lu.ipiv != np.arange(n)) > 0
    assert np.allclose(lu.store, lub, rtol=0, atol=1e-12 * np.abs(lub).max())
    A = O.band_to_dense(ab, k)
    f = inputs.rhs(n, 2, seed=9)
    x = lu.solve(f)
    assert np.linalg.norm(x - np.linalg.solve(A, f)) <= 1e-12 * np.linalg.norm(x)
    xl, info = lapack.dgbtrs(lub, k, k, f, ipiv)
    assert np.linalg.norm(x - xl) <= 1e-13 * np.linalg.norm(x)
    xt = lu.solve(f, trans=True)
    assert np.linalg.norm(xt - np.linalg.solve(A.T, f)) <= 1e-12 * np.linalg.norm(xt)


def test_zero_pivot_is_reported():
    ab = inputs.dominant_band(20, 2, 1.5, seed=1)
    ab[2, 5] = 0.0          # A[5,5] = 0 -> elimination hits it unless fill changes it
    ab[:, 5] = 0.0          # whole column 5 zero: singular whichever way
    with pytest.raises(O.SingularPivot):
        O.BandLU(ab, 2, pivoting=False)
    with pytest.raises(O.SingularPivot):
        O.BandLU(ab, 2, pivoting=True)


def test_dominance_generator_definition():
    ab = inputs.dominant_band(30, 4, 1.5, seed=2)
    A = O.band_to_dense(ab, 4)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert np.allclose(np.diag(A), 1.5 * off)
    assert np.all(np.abs(A[np.abs(np.subtract.outer(np.arange(30), np.arange(30))) > 4]) == 0)
