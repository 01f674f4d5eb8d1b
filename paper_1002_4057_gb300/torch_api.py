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
           wait_timeout_s=0.0, fault_drop_task=-1, residual=0, refine_order=0, variant=0, split_segment=0,
           diag_fp64=0):
    """In place: lower triangle of A <- lower triangle of A^{-1} (Steps 1-3).
    Mixed precision (precision=1): refine_steps corrections of order
    refine_order (0 = 2); diag_fp64=1 runs the DAG's diagonal POTRF/TRTRI in
    FP64.  variant: an execution variant of the FP64 plan
    (SPDINV_VARIANT_*; split_segment for SPDINV_VARIANT_SPLIT3)."""
    n, lda = _lda(A, torch.float64)
    info = _info_buf(A.device) if info is None else info
    if (tile or ctas_per_sm or precision or refine_steps or wait_timeout_s or fault_drop_task >= 0 or residual
            or refine_order or variant or split_segment or diag_fp64):
        o = L.spdinv_opts(tile, ctas_per_sm, precision, refine_steps, float(wait_timeout_s), fault_drop_task,
                          residual, refine_order, variant, split_segment, diag_fp64)
        st = L.spdinv_potri_ex(n, A.data_ptr(), lda, o, info.data_ptr(), _stream(stream))
        _check(st, "spdinv_potri_ex")
    else:
        _check(L.spdinv_potri(n, A.data_ptr(), lda, info.data_ptr(), _stream(stream)), "spdinv_potri")
    return info


def inverse_diag(A, info=None, stream=None):
    """diag(A^{-1}) of an SPD matrix (column-major float64 CUDA tensor; only
    its lower triangle is read, nothing is written) as a new length-n
    tensor: Steps 1 and 2 and the diagonal tiles of Step 3."""
    n, lda = _lda(A, torch.float64)
    info = _info_buf(A.device) if info is None else info
    d = torch.empty(n, dtype=torch.float64, device=A.device)
    _check(L.spdinv_potri_diag(n, A.data_ptr(), lda, d.data_ptr(), info.data_ptr(), _stream(stream)),
           "spdinv_potri_diag")
    return d


def potri_noalloc_(A, info=None, stream=None):
    """potri_ (FP64, tile 32) without any device allocation by the library,
    for n <= SPDINV_NOALLOC_MAX_N; calls must not overlap on the GPU."""
    n, lda = _lda(A, torch.float64)
    info = _info_buf(A.device) if info is None else info
    _check(L.spdinv_potri_noalloc(n, A.data_ptr(), lda, info.data_ptr(), _stream(stream)), "spdinv_potri_noalloc")
    return info


def inverse_residual(A, X, residual=L.SPDINV_RESIDUAL_EMULATED, stream=None):
    """R = I - A X as a new column-major n x n float64 tensor, for a
    symmetric A given by its lower triangle (column-major) and a full X
    (column-major, leading dimension n).  residual selects how the product
    is formed (SPDINV_RESIDUAL_*)."""
    n, lda = _lda(A, torch.float64)
    nx, ldx = _lda(X, torch.float64)
    if nx != n or ldx != max(n, 1) or X.device != A.device:
        raise ValueError("X must be n x n on A's device, column-major with leading dimension n")
    R = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    _check(L.spdinv_inverse_residual(n, A.data_ptr(), lda, X.data_ptr(), R.data_ptr(), int(residual),
                                     _stream(stream)), "spdinv_inverse_residual")
    return R


# ------------------------------------------------------- caller workspace
_workspaces = {}  # device index -> the caller's buffer, kept alive while set


def workspace_size(n, routine=L.SPDINV_ROUTINE_POTRI, tile=0, precision=0, refine_steps=0, residual=0,
                   refine_order=0):
    """Bytes of device workspace one call of `routine` on an order-n matrix
    uses (the options as for potri_)."""
    o = L.spdinv_opts(tile, 0, precision, refine_steps, 0.0, -1, residual, refine_order)
    st, nbytes = L.spdinv_workspace_size(n, routine, o)
    _check(st, "spdinv_workspace_size")
    return nbytes


def set_workspace(buf, device=None):
    """Make the single-matrix calls on buf's device use `buf` (a contiguous
    CUDA tensor; its bytes, from a 256-byte aligned start) as their
    workspace, so that they allocate nothing; None returns `device`'s
    (default: the current device's) calls to the library's own workspace.
    The tensor is kept alive here until it is replaced."""
    if buf is None:
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(dev):
            _check(L.spdinv_set_workspace(None, 0), "spdinv_set_workspace")
        _workspaces.pop(dev.index, None)
        return
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    with torch.cuda.device(buf.device):
        _check(L.spdinv_set_workspace(buf.data_ptr(), buf.numel() * buf.element_size()), "spdinv_set_workspace")
    _workspaces[buf.device.index] = buf


# ---------------------------------------------------------------- batched
class PreparedBatch:
    """The host size arrays and the device pointer array of a batch of
    column-major matrices (float64 or float32), kept alive so that repeated
    calls -- including calls captured in a CUDA graph -- need no host work
    beyond the launch.  Call run() once outside capture first: the first call
    with a new size list builds and uploads its plan."""

    def __init__(self, mats):
        import numpy as np
        if not mats:
            raise ValueError("empty batch")
        self.dtype = mats[0].dtype
        if self.dtype not in (torch.float64, torch.float32):
            raise ValueError("float64 or float32 matrices expected")
        dev = mats[0].device
        ns, ldas, ptrs = [], [], []
        for M in mats:
            n, lda = _lda(M, self.dtype)
            if M.device != dev:
                raise ValueError("all matrices must be on one device")
            ns.append(n)
            ldas.append(lda)
            ptrs.append(M.data_ptr())
        self.mats = list(mats)
        self.h_n = np.ascontiguousarray(ns, dtype=np.int32)
        self.h_lda = np.ascontiguousarray(ldas, dtype=np.int32)
        self.d_ptrs = torch.tensor(ptrs, dtype=torch.int64, device=dev)
        self.info = torch.zeros(len(mats), dtype=torch.int32, device=dev)

    def run(self, stream=None):
        fn = L.spdinv_potri_batched if self.dtype == torch.float64 else L.spdinv_spotri_batched
        st = fn(len(self.mats), self.h_n.ctypes.data, self.d_ptrs.data_ptr(), self.h_lda.ctypes.data,
                self.info.data_ptr(), _stream(stream))
        _check(st, "spdinv_(s)potri_batched")
        return self.info


def potri_batched_(mats, stream=None):
    """In place on every matrix of the list (column-major float64/float32
    CUDA tensors of any sizes): lower triangle <- lower triangle of its
    inverse, in one launch.  Returns the per-matrix info tensor."""
    return PreparedBatch(mats).run(stream)


# ---------------------------------------------------------------- autograd
def _as_batch(A):
    if A.dim() == 2:
        return A.unsqueeze(0), True
    if A.dim() == 3:
        return A, False
    raise ValueError("expected (n, n) or (batch, n, n)")


def _batched_views(buf):
    """Column-major views of each matrix of a contiguous (batch, n, n) buffer
    holding the matrices transposed (buf[k] row-major = A_k column-major)."""
    return [buf[k].t() for k in range(buf.shape[0])]


class SpdInverse(torch.autograd.Function):
    """X = A^{-1} for symmetric positive definite A (float64 or float32,
    (n, n) or (batch, n, n)), with grad_A = -sym(X G X) in the backward.

    Forward: the batched inversion (lower triangles) and a mirror kernel that
    completes the symmetric X; backward: the grad kernel.  All arithmetic in
    libspdinv.so."""

    @staticmethod
    def forward(ctx, A):
        A3, squeeze = _as_batch(A)
        if not A3.is_cuda:
            raise ValueError("CUDA tensor expected")
        b, n, _ = A3.shape
        buf = A3.detach().transpose(-1, -2).contiguous()  # column-major copies
        info = PreparedBatch(_batched_views(buf)).run()
        s = _stream(None)
        mirror = L.spdinv_mirror_lower if buf.dtype == torch.float64 else L.spdinv_smirror_lower
        _check(mirror(b, n, buf.data_ptr(), max(n, 1), n * n, s), "spdinv_mirror_lower")
        ctx.save_for_backward(buf)
        ctx.info = info
        ctx.squeeze = squeeze
        return buf[0] if squeeze else buf

    @staticmethod
    def backward(ctx, G):
        (X,) = ctx.saved_tensors
        G3 = (G.unsqueeze(0) if ctx.squeeze else G).contiguous()
        b, n, _ = X.shape
        grad = torch.empty_like(X)
        fn = L.spdinv_potri_backward if X.dtype == torch.float64 else L.spdinv_spotri_backward
        # X, sym(G) and grad are symmetric, so the row-/column-major reading of
        # their buffers does not matter.
        st = fn(b, n, X.data_ptr(), max(n, 1), n * n, G3.data_ptr(), max(n, 1), n * n,
                grad.data_ptr(), max(n, 1), n * n, _stream(None))
        _check(st, "spdinv_potri_backward")
        return grad[0] if ctx.squeeze else grad


def spd_inverse(A):
    """Differentiable A^{-1} of SPD matrices (see SpdInverse)."""
    return SpdInverse.apply(A)


TRACE_DTYPE = [("task", "<u4"), ("sm", "<u4"), ("ticket", "<u4"), ("cta", "<u4"), ("t_start_ns", "<u8"),
               ("t_end_ns", "<u8"), ("t_wait_ns", "<u8"), ("reserved", "<u8")]
TRACE_RECORD_BYTES = 48


def traced_potri_(A, capacity=None, **kw):
    """potri_ with the per-task trace on: returns (info, records), records a
    numpy structured array (TRACE_DTYPE) indexed by ticket.  The buffer is
    sized from the plan's task count (spdinv_plan_tasks) unless given."""
    import numpy as np
    n, _ = _lda(A, torch.float64)
    if capacity is None:
        tile = kw.get("tile", 0) or (32 if n <= 16384 else 64)
        st, tasks, _ = L.spdinv_plan_tasks(max(n, 1), tile, 0)
        _check(st, "spdinv_plan_tasks")
        capacity = max(len(tasks), 1) + 4096  # room for a split variant's segments
    buf = torch.zeros(capacity * TRACE_RECORD_BYTES, dtype=torch.uint8, device=A.device)
    _check(L.spdinv_set_trace(buf.data_ptr(), capacity), "spdinv_set_trace")
    try:
        info = potri_(A, **kw)
        torch.cuda.synchronize(A.device)
    finally:
        L.spdinv_set_trace(None, 0)
    rec = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=np.dtype(TRACE_DTYPE))
    return info, rec
