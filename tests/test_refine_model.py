"""A numpy model of the mixed-precision correction's arithmetic: balanced
base-256 digits of row/column-scaled operands, exact products of digit pairs,
levels s + t kept up to a limit.  It is the model that fixed the library's
level limits (7 for the last residual R = I - A X, and 4, 3, 2, ... for the
terms X R^m of an order-p step); these tests pin the properties the design
relies on.  It shares nothing with the CUDA path (which tests/test_gpu_mixed.py
checks against the FP64 oracle) and is not part of the oracle."""
import numpy as np
import pytest

import spd_inputs as si

CHAIN = [4, 3, 2, 2, 1, 1, 1]  # level limit of X R^m, m = 1..7


def expo(m):
    """e with 2^e > 2 m (0 for m = 0)."""
    _, e = np.frexp(m)
    return np.where(m > 0, e + 1, 0)


def digits(M, e, S):
    """S balanced base-256 digits of each row of M scaled by 2^-e_row."""
    u = np.ldexp(M, -e[:, None])
    out = []
    for _ in range(S):
        u = u * 256.0
        a = np.rint(u)
        u = u - a
        out.append(a)
    return out


def product(Lm, Rm, S, L):
    """Lm @ Rm from S digits of Lm's rows and of Rm's columns, levels <= L."""
    e = expo(np.abs(Lm).max(axis=1))
    f = expo(np.abs(Rm).max(axis=0))
    a, b = digits(Lm, e, S), digits(Rm.T, f, S)
    P = np.zeros((Lm.shape[0], Rm.shape[1]))
    for lv in range(L + 1):
        acc = np.zeros_like(P)
        for s in range(lv + 1):
            if s < S and lv - s < S:
                acc += a[s] @ b[lv - s].T  # integers: exact in FP64 at these sizes
        P += np.ldexp(acc, -8 * (lv + 2))
    return np.ldexp(np.ldexp(P, e[:, None]), f[None, :])


def correction(A, X, order, last_levels=7):
    """One step X (I + R + ... + R^{p-1}), R = I - A X, the terms as
    (X R^{m-1}) R, symmetric, from fewer digits as they shrink."""
    n = A.shape[0]
    R = np.eye(n) - product(A, X, 7, last_levels)
    Y, out = X, X.copy()
    for L in CHAIN[:order - 1]:
        Y = product(Y, R, L + 1, L)
        Y = np.tril(Y) + np.tril(Y, -1).T
        out += Y
    return out


def fp32_inverse(A):
    import scipy.linalg as sl
    c, info = sl.lapack.spotrf(A.astype(np.float32), lower=1)
    assert info == 0
    x, info = sl.lapack.spotri(c, lower=1)
    assert info == 0
    X = np.tril(x).astype(np.float64)
    return X + np.tril(X, -1).T


def relerr(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


def test_digits_are_exact_bf16_integers_and_chunks_fit_fp32():
    r = np.random.default_rng(3)
    M = r.standard_normal((64, 64)) * np.exp(r.uniform(-20, 20, size=(64, 1)))
    e = expo(np.abs(M).max(axis=1))
    ds = digits(M, e, 7)
    for d in ds:
        assert np.all(np.abs(d) <= 128) and np.all(d == np.rint(d))
    # the digits reconstruct the value to 2^-56 of the row scale
    back = sum(np.ldexp(d, -8 * (s + 1)) for s, d in enumerate(ds))
    assert np.all(np.abs(np.ldexp(M, -e[:, None]) - back) <= 2.0 ** -57)
    # a 1024-deep chunk of digit products is at most 2^24: exact in an FP32 accumulator
    assert 1024 * 128 * 128 == 2 ** 24


def test_emulated_residual_matches_fp64_product():
    A, _, _ = si.spectral_spd(256, 1e3, seed=11)
    X = fp32_inverse(A)
    R = np.eye(256) - product(A, X, 7, 7)
    Rref = np.eye(256) - A @ X
    scale = np.max(np.abs(A) @ np.abs(X))
    assert np.max(np.abs(R - Rref)) <= 1e-15 * scale


@pytest.mark.parametrize("cond,order,bound", [(1e2, 3, 1e-12), (1e4, 4, 1e-11)])
def test_one_step_of_order_p_reaches_the_target(cond, order, bound):
    n = 384
    A, Q, lam = si.spectral_spd(n, cond, seed=si.SEED_BASE + 2)
    Ainv = (Q / lam) @ Q.T
    X0 = fp32_inverse(A)
    e0 = relerr(X0, Ainv)
    e2 = relerr(correction(A, X0, 2), Ainv)
    ep = relerr(correction(A, X0, order), Ainv)
    # the FP32 start, one Newton-Schulz step, one step of order p
    assert e0 > 1e-7
    assert ep <= bound and ep < e2
