"""Closed-form inverses used to pin the oracle and, at sizes the oracle cannot
reach, as the oracle itself (sampled entries).  TEST INFRASTRUCTURE ONLY.

All indices are 0-based unless a docstring says otherwise.
"""
from fractions import Fraction

import numpy as np


def tridiag_cholesky(n):
    """Cholesky factor of T = tridiag(-1, 2, -1) (order n).

    With 1-based i: L_ii = sqrt((i+1)/i), L_{i+1,i} = -sqrt(i/(i+1)).
    (Check: L_11^2 = 2; L_{i+1,i}^2 + L_{i+1,i+1}^2 = i/(i+1) + (i+2)/(i+1) = 2;
    L_{i+1,i} L_ii = -1.)
    """
    i = np.arange(1, n + 1, dtype=np.float64)
    L = np.zeros((n, n), order="F")
    L[np.arange(n), np.arange(n)] = np.sqrt((i + 1) / i)
    L[np.arange(1, n), np.arange(n - 1)] = -np.sqrt(i[:-1] / (i[:-1] + 1))
    return L


def tridiag_cholesky_inverse(n):
    """(L^{-1})_ij = j / sqrt(i (i+1)) for i >= j (1-based), L as above."""
    i = np.arange(1, n + 1, dtype=np.float64)[:, None]
    j = np.arange(1, n + 1, dtype=np.float64)[None, :]
    return np.asfortranarray(np.where(i >= j, j / np.sqrt(i * (i + 1)), 0.0))


def tridiag_inverse_entries(n, rows, cols):
    """(T^{-1})_ij = min(i,j) (n+1-max(i,j)) / (n+1), 1-based i, j.

    rows/cols are 0-based index arrays.
    """
    i = np.asarray(rows, dtype=np.float64) + 1
    j = np.asarray(cols, dtype=np.float64) + 1
    return np.minimum(i, j) * (n + 1 - np.maximum(i, j)) / (n + 1)


def tridiag_inverse(n):
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.asfortranarray(tridiag_inverse_entries(n, r, c))


def bidiag_inverse_entries(s, rows, cols):
    """Exact A^{-1} entries for A = L L^T, L = I + diag(s, -1), s_k in {+1,-1}.

    X = L^{-1} has X_ij = prod_{k=j}^{i-1} (-s_k) for i >= j, and
    (A^{-1})_ij = sum_{k >= max(i,j)} X_ki X_kj = (n - max(i,j)) X_{max,min}
    (0-based), since X_ki X_kj = X_ki^2 X_ij = X_ij for k >= i >= j.
    Integers of magnitude <= n.
    """
    s = np.asarray(s, dtype=np.int64)
    n = s.size + 1
    # prefix products p_m = prod_{k<m} (-s_k); X_ij = p_i / p_j = p_i * p_j
    p = np.ones(n, dtype=np.int64)
    p[1:] = np.cumprod(-s)
    r = np.asarray(rows, dtype=np.int64)
    c = np.asarray(cols, dtype=np.int64)
    hi = np.maximum(r, c)
    lo = np.minimum(r, c)
    return ((n - hi) * p[hi] * p[lo]).astype(np.float64)


def bidiag_inverse(s):
    n = len(s) + 1
    r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.asfortranarray(bidiag_inverse_entries(s, r, c))


def exact_inverse_rational(M):
    """Exact inverse of a small nonsingular rational/integer matrix by
    Gauss-Jordan elimination over Fractions (brute force, tiny n only)."""
    n = len(M)
    a = [[Fraction(M[i][j]) for j in range(n)] + [Fraction(int(i == j)) for j in range(n)]
         for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        piv = a[c][c]
        a[c] = [v / piv for v in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [vr - f * vc for vr, vc in zip(a[r], a[c])]
    return [row[n:] for row in a]


def hilbert(n):
    """H_ij = 1/(i+j-1), 1-based, as exact Fractions."""
    return [[Fraction(1, i + j + 1) for j in range(n)] for i in range(n)]


def hilbert_inverse_exact(n):
    """Integer inverse of the order-n Hilbert matrix (exact rationals)."""
    inv = exact_inverse_rational(hilbert(n))
    out = np.zeros((n, n), dtype=object)
    for i in range(n):
        for j in range(n):
            assert inv[i][j].denominator == 1
            out[i, j] = int(inv[i][j])
    return out


def adjugate3(M):
    """Exact inverse of a 3x3 integer matrix as adj(M)/det(M) (Fractions)."""
    m = [[int(M[i][j]) for j in range(3)] for i in range(3)]

    def minor(i, j):
        r = [x for x in range(3) if x != i]
        c = [y for y in range(3) if y != j]
        return m[r[0]][c[0]] * m[r[1]][c[1]] - m[r[0]][c[1]] * m[r[1]][c[0]]

    det = sum(((-1) ** j) * m[0][j] * minor(0, j) for j in range(3))
    return [[Fraction(((-1) ** (i + j)) * minor(j, i), det) for j in range(3)] for i in range(3)]


def spectral_inverse_columns(Q, lam, cols):
    """Columns of (Q diag(lam) Q^T)^{-1} = Q diag(1/lam) Q^T, O(n^2) each."""
    Q = np.asarray(Q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    cols = np.asarray(cols)
    return Q @ (Q[cols, :].T / lam[:, None])
