"""FP64 CPU oracle for tiled SPD inversion -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline and
reference legs) may import this package.  The CUDA path never does, and this
package imports nothing from it.

Each function states the passage of Agullo et al. (Sec. 2, Algorithm 1) or
the mathematical definition it follows.  Matrices are numpy float64 arrays in
Fortran (column-major) order, so that M[i, j] is row i, column j of the
column-major buffer the C routines see; only the lower triangle is used.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None
EPS = 2.0 ** -53  # LAPACK dlamch('E'): unit roundoff of IEEE double


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        for name in ("oracle_potf2", "oracle_trti2", "oracle_lauu2", "oracle_potri"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
            f.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def _run(name, M):
    M = np.array(M, dtype=np.float64, order="F", copy=True)
    n = M.shape[0]
    assert M.ndim == 2 and M.shape[1] == n
    info = getattr(_load(), name)(n, M.ctypes.data, max(n, 1))
    return M, int(info)


def potrf(A):
    """Step 1 (Sec. 2, Algorithm 1): Cholesky factor L of A = L L^T, lower.

    Returns (M, info): M's lower triangle holds L, its strictly upper part is
    A's untouched; info = j+1 for the first non-positive (or NaN) pivot.
    """
    return _run("oracle_potf2", A)


def trtri(L):
    """Step 2 (Sec. 2, Algorithm 1): X = L^{-1} for lower non-unit L.

    info = j+1 for the first exactly-zero diagonal entry (matrix unchanged).
    """
    return _run("oracle_trti2", L)


def lauum(X):
    """Step 3 (Sec. 2, Algorithm 1): lower triangle of X^T X."""
    M, _ = _run("oracle_lauu2", X)
    return M


def potri(A):
    """Steps 1-3 (Algorithm 1): lower triangle of A^{-1}; (M, info)."""
    return _run("oracle_potri", A)


def lower(M):
    """The lower triangle of M (upper part zeroed)."""
    return np.tril(np.asarray(M))


def symmetrize_lower(M):
    """Full symmetric matrix from a lower triangle: tril(M) + tril(M, -1)^T."""
    Lo = np.tril(np.asarray(M, dtype=np.float64))
    return Lo + np.tril(Lo, -1).T


def lapack_ratio(A, X):
    """LAPACK inverse test ratio ||I - A X||_1 / (n ||A||_1 ||X||_1 eps).

    A and X are full symmetric matrices; eps = 2^-53.
    """
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = A.shape[0]
    R = np.eye(n) - A @ X
    return float(np.linalg.norm(R, 1) / (n * np.linalg.norm(A, 1) * np.linalg.norm(X, 1) * EPS))


def rel_frobenius(X, Y):
    """||X - Y||_F / ||Y||_F (full matrices)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def backward(X, G):
    """Gradient of f(A) = <G, A^{-1}> over symmetric A, with X = A^{-1}.

    d(A^{-1}) = -X dA X, so <G, d(A^{-1})> = <-X G X, dA> for symmetric X;
    restricted to symmetric directions the gradient is -sym(X G X) =
    -(X G X + (X G X)^T)/2.
    """
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    M = X @ G @ X
    return -(M + M.T) / 2.0
