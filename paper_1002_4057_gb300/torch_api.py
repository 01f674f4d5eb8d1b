"""Torch-tensor wrappers over the C-ABI (marshalling only).

Matrices are column-major CUDA tensors: shape (n, n) with stride (1, lda),
e.g. ``M.t()`` of a row-major tensor, or ``colmajor(M)``.  Every step of the
computation runs in libspdinv.so; torch supplies device memory and streams.
"""
import torch

from . import _lib as L


class SpdinvError(RuntimeError):
    pass


def _check(st, what):
    if st != L.SPDINV_OK:
        msg = L.STATUS_NAMES.get(st, str(st))
        if st == L.SPDINV_ERR_CUDA:
            msg += ": " + L.spdinv_last_cuda_error()
        raise SpdinvError("%s failed: %s" % (what, msg))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def colmajor(M):
    """A column-major copy of a square matrix (same dtype/device)."""
    return M.t().contiguous().t()


def _lda(A, dtype):
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("expected a square matrix")
    if A.dtype != dtype or not A.is_cuda:
        raise ValueError("expected a CUDA %s tensor" % dtype)
    n = A.shape[0]
    if n > 1 and A.stride(0) != 1:
        raise ValueError("expected a column-major tensor (stride (1, lda)); use colmajor()")
    return n, max(A.stride(1), max(n, 1)) if n > 1 else max(n, 1)


def _info_buf(device):
    return torch.zeros(1, dtype=torch.int32, device=device)


def potrf_(A, info=None, stream=None):
    """In place: lower triangle of A <- L (Step 1).  Returns the device info tensor."""
    n, lda = _lda(A, torch.float64)
    info = _info_buf(A.device) if info is None else info
    _check(L.spdinv_potrf(n, A.data_ptr(), lda, info.data_ptr(), _stream(stream)), "spdinv_potrf")
    return info


def trtri_(A, info=None, stream=None):
    """In place: lower triangle of A <- L^{-1} (Step 2)."""
    n, lda = _lda(A, torch.float64)
    info = _info_buf(A.device) if info is None else info
    _check(L.spdinv_trtri(n, A.data_ptr(), lda, info.data_ptr(), _stream(stream)), "spdinv_trtri")
    return info


def lauum_(A, stream=None):
    """In place: lower triangle of A <- X^T X (Step 3)."""
    n, lda = _lda(A, torch.float64)
    _check(L.spdinv_lauum(n, A.data_ptr(), lda, _stream(stream)), "spdinv_lauum")


def potri_(A, info=None, stream=None, tile=0, ctas_per_sm=0, precision=0, refine_steps=0,
           wait_timeout_s=0.0, fault_drop_task=-1):
    """In place: lower triangle of A <- lower triangle of A^{-1} (Steps 1-3)."""
    n, lda = _lda(A, torch.float64)
    info = _info_buf(A.device) if info is None else info
    if tile or ctas_per_sm or precision or refine_steps or wait_timeout_s or fault_drop_task >= 0:
        o = L.spdinv_opts(tile, ctas_per_sm, precision, refine_steps, float(wait_timeout_s), fault_drop_task)
        st = L.spdinv_potri_ex(n, A.data_ptr(), lda, o, info.data_ptr(), _stream(stream))
        _check(st, "spdinv_potri_ex")
    else:
        _check(L.spdinv_potri(n, A.data_ptr(), lda, info.data_ptr(), _stream(stream)), "spdinv_potri")
    return info


def mirror_lower(A):
    """Full symmetric matrix from the lower triangle (a new tensor)."""
    Lo = torch.tril(A)
    return Lo + torch.tril(Lo, -1).t()
