"""Seeded synthetic inputs for SPD inversion: the only module shared by the
oracle's checks and the CUDA path's tests and benchmark.

It builds test matrices and holds none of the inversion arithmetic.  Every
generator draws from numpy's PCG64 (``default_rng(seed)``) so that the same
seed gives the same bits on every machine; seeds default to
SEED_BASE + workload index.  Matrices are float64, Fortran (column-major)
order, exactly symmetric.

Workloads (the shapes of the paper's experiments, Sec. 2-3: dense SPD
matrices, plus the added batched and differentiable forms):
  0  n=512, lam log-uniform in [1, 1e3]              (+ tridiag(-1,2,-1))
  1  n=4096 / 16384, lam log-uniform in [1, 1e4]
  2  n=16384 / 32768, cond in {1e2, 1e4, 1e6}        (mixed precision)
  3  4096 matrices, n ~ U{16..256}, A = B B^T/n + 0.1 I
  4  256 matrices, n=512, A = B B^T/n + I, G = sym(N(0,1))
"""
import numpy as np

SEED_BASE = 1002405700


def rng(seed):
    return np.random.default_rng(seed)


def log_uniform_spectrum(n, cond, seed):
    """n eigenvalues, log-uniform in [1, cond], with lam_0 = 1 and
    lam_{n-1} = cond forced so that cond(A) = cond exactly (n >= 2)."""
    r = rng(seed + 7919)
    lam = np.exp(np.sort(r.uniform(0.0, np.log(cond), size=n)))
    lam[0] = 1.0
    if n > 1:
        lam[-1] = float(cond)
    return lam


def orthogonal(n, seed, device=None):
    """Q from the QR factorisation of a seeded N(0,1) n x n matrix.

    The Gaussian is always drawn on the host (same bits everywhere); the QR
    runs in numpy, or in torch on ``device`` for large n.  Returns a numpy
    Fortran array, or a torch tensor on ``device`` when one is given.
    """
    g = rng(seed).standard_normal((n, n))
    if device is None:
        q, _ = np.linalg.qr(g)
        return np.asfortranarray(q)
    import torch
    gt = torch.from_numpy(g).to(device)
    del g
    q, _ = torch.linalg.qr(gt)
    return q


def spectral_spd(n, cond, seed, device=None):
    """A = Q diag(lam) Q^T (made exactly symmetric), its Q and lam.

    With ``device`` (a torch device), A and Q are torch tensors there
    (column-major order is irrelevant for a symmetric A)."""
    lam = log_uniform_spectrum(n, cond, seed)
    Q = orthogonal(n, seed, device)
    if device is None:
        A = (Q * lam) @ Q.T
        A = 0.5 * (A + A.T)
        return np.asfortranarray(A), Q, lam
    import torch
    lt = torch.from_numpy(lam).to(Q.device)
    A = (Q * lt) @ Q.T
    A = 0.5 * (A + A.T)
    # A is exactly symmetric: its transpose is the column-major view of it
    return A.t(), Q, lam


def tridiag(n):
    """T = tridiag(-1, 2, -1) of order n."""
    T = np.zeros((n, n), order="F")
    idx = np.arange(n)
    T[idx, idx] = 2.0
    T[idx[1:], idx[:-1]] = -1.0
    T[idx[:-1], idx[1:]] = -1.0
    return T


def bidiag_signs(n, seed):
    """Signs s_k in {+1, -1}, k = 0..n-2, for L = I + diag(s, -1)."""
    return rng(seed).choice(np.array([-1, 1], dtype=np.int64), size=max(n - 1, 0))


def bidiag_integer_spd(n, seed):
    """Integer SPD A = L L^T with L = I + diag(s, -1): A_00 = 1, A_ii = 2
    (i > 0), A_{i+1,i} = A_{i,i+1} = s_i.  Returns (A, s)."""
    s = bidiag_signs(n, seed)
    A = np.zeros((n, n), order="F")
    idx = np.arange(n)
    A[idx, idx] = 2.0
    if n:
        A[0, 0] = 1.0
    A[idx[1:], idx[:-1]] = s
    A[idx[:-1], idx[1:]] = s
    return A, s


def wishart_spd(n, shift, seed):
    """A = B B^T / n + shift I with B ~ N(0,1) n x n."""
    B = rng(seed).standard_normal((n, n))
    A = B @ B.T / n + shift * np.eye(n)
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A)


def batch_sizes(count, lo, hi, seed):
    """count sizes drawn uniformly from {lo, ..., hi}."""
    return rng(seed).integers(lo, hi + 1, size=count).astype(np.int64)


def wishart_batch(sizes, shift, seed):
    """One Wishart SPD matrix per size, each from its own seeded stream."""
    return [wishart_spd(int(n), shift, seed * 100003 + k) for k, n in enumerate(sizes)]


def symmetric_gaussian(n, seed):
    """G = (M + M^T)/2 with M ~ N(0,1)."""
    M = rng(seed).standard_normal((n, n))
    return np.asfortranarray(0.5 * (M + M.T))


def integer_spd3(seed):
    """A seeded 3x3 integer SPD matrix: M^T M + I with M in {-3..3}^{3x3}."""
    M = rng(seed).integers(-3, 4, size=(3, 3))
    return (M.T @ M + np.eye(3, dtype=np.int64)).astype(np.int64)
