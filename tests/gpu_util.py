"""Helpers for the GPU tests: move seeded numpy inputs to column-major CUDA
tensors and read lower triangles back.  No arithmetic of the method here."""
import numpy as np


def to_dev(A, dev, lda=None):
    """Column-major CUDA float64 copy of A (optionally with lda > n)."""
    import torch
    A = np.asfortranarray(A, dtype=np.float64)
    n = A.shape[0]
    if lda is None or lda == n:
        return torch.from_numpy(A).to(dev)
    store = torch.full((n * lda,), float("nan"), dtype=torch.float64)
    view = store.as_strided((n, n), (1, lda))
    view.copy_(torch.from_numpy(A))
    return store.to(dev).as_strided((n, n), (1, lda))


def lower_np(dA):
    return np.tril(dA.cpu().numpy())


def full_from_lower(M):
    Lo = np.tril(np.asarray(M))
    return Lo + np.tril(Lo, -1).T
