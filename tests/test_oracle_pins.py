"""Pins for the FP64 CPU oracle: each check compares it with something other
than itself (closed forms, exact rational arithmetic, exact integer cases,
LAPACK through scipy, finite differences)."""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import oracle
from oracle import closed_forms as cf
import spd_inputs as si

EPS = 2.0 ** -53


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_tridiag_inverse_closed_form_is_exact(n):
    T = si.tridiag(n)
    exact = cf.exact_inverse_rational([[int(v) for v in row] for row in T])
    got = cf.tridiag_inverse(n)
    for i in range(n):
        for j in range(n):
            assert abs(got[i, j] - float(exact[i][j])) <= 1e-15


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_tridiag_factor_closed_forms(n):
    L = cf.tridiag_cholesky(n)
    assert np.allclose(L @ L.T, si.tridiag(n), atol=1e-14, rtol=0)
    X = cf.tridiag_cholesky_inverse(n)
    assert np.allclose(X @ L, np.eye(n), atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 10])
def test_bidiag_closed_form_is_exact(n):
    A, s = si.bidiag_integer_spd(n, seed=11 + n)
    exact = cf.exact_inverse_rational([[int(v) for v in row] for row in A])
    got = cf.bidiag_inverse(s)
    for i in range(n):
        for j in range(n):
            assert got[i, j] == float(exact[i][j])


def test_hilbert_inverse_integer_and_known_value():
    # The inverse of the order-3 Hilbert matrix is a textbook value.
    inv3 = cf.hilbert_inverse_exact(3)
    assert inv3.tolist() == [[9, -36, 30], [-36, 192, -180], [30, -180, 180]]


# -------------------------------------------------------------- step 1 (potf2)
@pytest.mark.parametrize("n", [1, 2, 64, 513])
def test_potrf_tridiag(n):
    L, info = oracle.potrf(si.tridiag(n))
    assert info == 0
    err = np.max(np.abs(np.tril(L) - cf.tridiag_cholesky(n)))
    assert err <= 64 * EPS  # rounding carried through the recurrence; a dropped term is O(1)


def test_potrf_residual_dense():
    A, _, _ = si.spectral_spd(300, 1e4, seed=5)
    L, info = oracle.potrf(A)
    assert info == 0
    L = np.tril(L)
    r = np.linalg.norm(A - L @ L.T, 1) / (300 * np.linalg.norm(A, 1) * EPS)
    assert r < 10


def test_potrf_matches_lapack():
    A, _, _ = si.spectral_spd(257, 1e3, seed=6)
    L, info = oracle.potrf(A)
    Lr, inf2 = lapack.dpotrf(A, lower=1, clean=1)
    assert info == 0 and inf2 == 0
    assert np.max(np.abs(np.tril(L) - Lr)) <= 1e-13 * np.max(np.abs(Lr))


@pytest.mark.parametrize("A,expect", [
    (np.diag([1.0, 2.0, -1.0, 3.0]), 3),
    (np.array([[1.0, 2.0], [2.0, 1.0]]), 2),
    (np.zeros((3, 3)), 1),
    (np.array([[4.0, 1.0], [1.0, np.nan]]), 2),
])
def test_potrf_info_first_failing_column(A, expect):
    _, info = oracle.potrf(A)
    assert info == expect
    _, info2 = oracle.potri(A)
    assert info2 == expect


# -------------------------------------------------------------- step 2 (trti2)
@pytest.mark.parametrize("n", [1, 2, 64, 300])
def test_trtri_tridiag_factor(n):
    X, info = oracle.trtri(cf.tridiag_cholesky(n))
    assert info == 0
    ref = cf.tridiag_cholesky_inverse(n)
    assert np.max(np.abs(np.tril(X) - ref)) <= 8 * n * EPS


def test_trtri_dense_identity():
    A, _, _ = si.spectral_spd(200, 1e2, seed=8)
    L, _ = oracle.potrf(A)
    L = np.tril(L)
    X, info = oracle.trtri(L)
    assert info == 0
    X = np.tril(X)
    r = np.linalg.norm(L @ X - np.eye(200), 1) / (200 * np.linalg.norm(L, 1) * np.linalg.norm(X, 1) * EPS)
    assert r < 10
    Xr, inf2 = lapack.dtrtri(L, lower=1)
    assert inf2 == 0
    assert np.max(np.abs(X - np.tril(Xr))) <= 1e-12 * np.max(np.abs(Xr))


def test_trtri_zero_diagonal_info():
    L = np.tril(np.ones((4, 4)))
    L[2, 2] = 0.0
    X, info = oracle.trtri(L)
    assert info == 3
    assert np.array_equal(X, L)


# -------------------------------------------------------------- step 3 (lauu2)
@pytest.mark.parametrize("n", [1, 2, 64, 300])
def test_lauum_tridiag(n):
    M = oracle.lauum(cf.tridiag_cholesky_inverse(n))
    ref = np.tril(cf.tridiag_inverse(n))
    assert np.max(np.abs(np.tril(M) - ref)) <= 4 * n * EPS * np.max(np.abs(ref))


def test_lauum_dense_vs_product():
    rng = np.random.default_rng(3)
    X = np.tril(rng.standard_normal((150, 150)))
    M = oracle.lauum(X)
    ref = X.T @ X
    assert np.max(np.abs(np.tril(M) - np.tril(ref))) <= 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------- whole potri
def test_potri_tridiag_512():
    n = 512
    M, info = oracle.potri(si.tridiag(n))
    assert info == 0
    ref = cf.tridiag_inverse(n)
    # cond(T) ~ 4(n+1)^2/pi^2 ~ 1.07e5
    assert oracle.rel_frobenius(oracle.symmetrize_lower(M), ref) < 1e-11


@pytest.mark.parametrize("n", [1, 2, 3, 17, 300])
def test_potri_integer_bidiag_bitwise(n):
    A, s = si.bidiag_integer_spd(n, seed=100 + n)
    M, info = oracle.potri(A)
    assert info == 0
    assert np.array_equal(np.tril(M), np.tril(cf.bidiag_inverse(s)))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_potri_hilbert_integer_inverse(n):
    H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    M, info = oracle.potri(H)
    assert info == 0
    exact = cf.hilbert_inverse_exact(n)
    got = np.rint(np.tril(M)).astype(np.int64)
    assert np.array_equal(got, np.tril(exact.astype(np.int64)))


@pytest.mark.parametrize("n", [7, 8])
def test_potri_hilbert_cond_scaled(n):
    H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)], order="F")
    M, info = oracle.potri(H)
    assert info == 0
    exact = cf.hilbert_inverse_exact(n).astype(np.float64)
    cond = np.linalg.cond(H)
    assert oracle.rel_frobenius(oracle.symmetrize_lower(M), exact) < 50 * cond * EPS


@pytest.mark.parametrize("seed", range(6))
def test_potri_adjugate_3x3(seed):
    A = si.integer_spd3(seed)
    exact = cf.adjugate3(A)
    M, info = oracle.potri(A.astype(np.float64))
    assert info == 0
    Ex = np.array([[float(v) for v in row] for row in exact])
    cond = np.linalg.cond(A.astype(np.float64))
    assert oracle.rel_frobenius(oracle.symmetrize_lower(M), Ex) < 20 * cond * EPS


@pytest.mark.parametrize("cond", [1e2, 1e4, 1e6])
def test_potri_lapack_ratio_and_scipy(cond):
    n = 512
    A, Q, lam = si.spectral_spd(n, cond, seed=si.SEED_BASE)
    M, info = oracle.potri(A)
    assert info == 0
    X = oracle.symmetrize_lower(M)
    assert oracle.lapack_ratio(A, X) <= 10
    # LAPACK dpotrf + dpotri through scipy: an independent library routine
    c, i1 = lapack.dpotrf(A, lower=1, clean=1)
    inv, i2 = lapack.dpotri(c, lower=1)
    assert i1 == 0 and i2 == 0
    ref = oracle.symmetrize_lower(inv)
    assert oracle.rel_frobenius(X, ref) < 50 * cond * EPS
    # spectral definition A^{-1} = Q diag(1/lam) Q^T on sampled columns
    cols = np.array([0, 1, n // 2, n - 1])
    colref = cf.spectral_inverse_columns(Q, lam, cols)
    assert np.linalg.norm(X[:, cols] - colref) / np.linalg.norm(colref) < 50 * cond * EPS


def test_exact_symmetry_of_symmetrized_output():
    A, _, _ = si.spectral_spd(100, 1e3, seed=9)
    M, _ = oracle.potri(A)
    X = oracle.symmetrize_lower(M)
    assert np.array_equal(X, X.T)


def test_upper_triangle_untouched():
    n = 50
    A, _, _ = si.spectral_spd(n, 1e2, seed=10)
    B = A.copy(order="F")
    iu = np.triu_indices(n, 1)
    B[iu] = 12345.0
    M, info = oracle.potri(B)
    assert info == 0
    assert np.all(M[iu] == 12345.0)
    M2, _ = oracle.potri(A)
    assert np.array_equal(np.tril(M), np.tril(M2))


def test_potri_is_composition_of_steps():
    A, _, _ = si.spectral_spd(97, 1e3, seed=12)
    L, _ = oracle.potrf(A)
    X, _ = oracle.trtri(L)
    M1 = oracle.lauum(X)
    M2, _ = oracle.potri(A)
    assert np.array_equal(np.tril(M1), np.tril(M2))


def test_n1_and_n0():
    M, info = oracle.potri(np.array([[4.0]]))
    assert info == 0 and M[0, 0] == 0.25
    M0, info0 = oracle.potri(np.zeros((0, 0)))
    assert info0 == 0 and M0.shape == (0, 0)


def test_thread_count_does_not_change_bits():
    A, _, _ = si.spectral_spd(160, 1e3, seed=13)
    t0 = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        M1, _ = oracle.potri(A)
        oracle.set_num_threads(max(t0, 2))
        M2, _ = oracle.potri(A)
    finally:
        oracle.set_num_threads(t0)
    assert np.array_equal(M1, M2)


# ------------------------------------------------------------------ backward
def test_backward_diagonal_closed_form():
    a = np.array([1.0, 2.0, 4.0, 0.5])
    X = np.diag(1.0 / a)
    G = si.symmetric_gaussian(4, seed=1)
    grad = oracle.backward(X, G)
    assert np.allclose(grad, -G / np.outer(a, a), rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [8, 16, 32])
def test_backward_finite_differences(n):
    A = si.wishart_spd(n, 1.0, seed=200 + n)
    G = si.symmetric_gaussian(n, seed=300 + n)
    E = si.symmetric_gaussian(n, seed=400 + n)

    def f(M):
        R, info = oracle.potri(M)
        assert info == 0
        return float(np.sum(G * oracle.symmetrize_lower(R)))

    h = 1e-5 * np.linalg.norm(A, 2)
    fd = (f(A + h * E) - f(A - h * E)) / (2 * h)
    X = oracle.symmetrize_lower(oracle.potri(A)[0])
    an = float(np.sum(oracle.backward(X, G) * E))
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


# ------------------------------------------------------------ error measures
# Each pin_* check takes the function under test, so that the mutant tests can
# run the same check against planted mistakes.
def pin_lapack_ratio(ratio):
    """A = diag(1, 2, 4), X = A^{-1} plus a in each entry of column 0
    (a = 2^-30, all exact): I - A X = -A E has column 0 = -(a, 2a, 4a), so
    ||I - A X||_1 = 7a; ||A||_1 = 4; ||X||_1 = 1 + 3a.  The ratio is
    7a / (3 * 4 * (1 + 3a) * 2^-53).  (X A instead of A X gives 3a, the
    infinity norm 4a, eps = 2^-52 half the value.)"""
    a = 2.0 ** -30
    A = np.diag([1.0, 2.0, 4.0])
    X = np.diag([1.0, 0.5, 0.25])
    X[:, 0] += a
    want = 7 * a / (3 * 4 * (1 + 3 * a) * 2.0 ** -53)
    assert ratio(A, X) == pytest.approx(want, rel=1e-12)


def pin_rel_frobenius(rel):
    """Y = 2 I_4 (||Y||_F = 4) and X = Y plus 1 in entry (0, 1): the error
    is 1/4; measured against X instead it would be 1/sqrt(17)."""
    Y = 2.0 * np.eye(4)
    X = Y.copy()
    X[0, 1] = 1.0
    assert rel(X, Y) == 0.25
    assert rel(Y, X) == pytest.approx(17 ** -0.5, rel=1e-15)


def pin_backward(backward):
    """Diagonal X = diag(1/a) and a non-symmetric G: (X G X)_ij = G_ij /
    (a_i a_j), so -sym(X G X)_ij = -(G_ij + G_ji) / (2 a_i a_j); the result
    is exactly symmetric.  Then finite differences of f(A) = <G, A^{-1}>
    along symmetric directions, which fix every symmetric gradient."""
    a = np.array([1.0, 2.0, 4.0, 0.5])
    G = si.rng(si.SEED_BASE + 40).standard_normal((4, 4))
    grad = backward(np.diag(1.0 / a), G)
    assert np.allclose(grad, -(G + G.T) / (2.0 * np.outer(a, a)), rtol=1e-15, atol=0)
    assert np.array_equal(grad, grad.T)
    n = 12
    A = si.wishart_spd(n, 1.0, seed=si.SEED_BASE + 41)
    G = si.rng(si.SEED_BASE + 42).standard_normal((n, n))
    X = oracle.symmetrize_lower(oracle.potri(A)[0])
    grad = backward(X, G)
    h = 1e-5 * np.linalg.norm(A, 2)
    for q in range(3):
        E = si.symmetric_gaussian(n, seed=si.SEED_BASE + 43 + q)
        fp = float(np.sum(G * oracle.symmetrize_lower(oracle.potri(A + h * E)[0])))
        fm = float(np.sum(G * oracle.symmetrize_lower(oracle.potri(A - h * E)[0])))
        an = float(np.sum(grad * E))
        assert abs((fp - fm) / (2 * h) - an) <= 1e-6 * max(1.0, abs(an))


def test_lapack_ratio_hand_value():
    pin_lapack_ratio(oracle.lapack_ratio)


def test_rel_frobenius_hand_value():
    pin_rel_frobenius(oracle.rel_frobenius)


def test_backward_nonsymmetric_gradient():
    pin_backward(oracle.backward)
