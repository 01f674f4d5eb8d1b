"""ctypes binding of libspdinv.so: the C-ABI functions under the same names.

Argument marshalling only.  The library is loaded from this package's lib/
folder (built by paper_1002_4057_gb300.build); there is no fallback: a
missing library raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libspdinv.so")

c_int64 = ctypes.c_int64
c_int = ctypes.c_int
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
P = ctypes.c_void_p  # device/host pointers and cudaStream_t are passed as integers

SPDINV_OK = 0
SPDINV_ERR_N = -1
SPDINV_ERR_LDA = -2
SPDINV_ERR_NULL = -3
SPDINV_ERR_CUDA = -4
SPDINV_ERR_TIMEOUT = -5
SPDINV_ERR_UNSUPPORTED = -6
SPDINV_ERR_WORKSPACE = -7

SPDINV_PREC_FP64 = 0
SPDINV_PREC_MIXED_FP32 = 1
SPDINV_PREC_MIXED_BF16X3 = 2
SPDINV_PREC_MIXED_TF32X3 = 3

SPDINV_NOALLOC_MAX_N = 1024

SPDINV_DEBUG_POISON = 1

SPDINV_PLAN_BOTTOM_LEVEL = 0
SPDINV_PLAN_ALAP = 1

SPDINV_ROUTINE_POTRI = 0
SPDINV_ROUTINE_POTRF = 1
SPDINV_ROUTINE_TRTRI = 2
SPDINV_ROUTINE_LAUUM = 3
SPDINV_ROUTINE_POTRI_DIAG = 4
SPDINV_ROUTINE_INVERSE_RESIDUAL = 5

SPDINV_RESIDUAL_EMULATED = 0
SPDINV_RESIDUAL_FP64 = 1
SPDINV_RESIDUAL_EMULATED_MMA_SYNC = 2

SPDINV_VARIANT_UUU = 1
SPDINV_VARIANT_SHARE_BC = 2
SPDINV_VARIANT_INPLACE = 4
SPDINV_VARIANT_SPLIT3 = 8

SPDINV_DAG_OUT_OF_PLACE = 1
SPDINV_DAG_RENAME_DIAG = 2
SPDINV_DAG_UUU = 4
SPDINV_DAG_PIPELINE = 8
SPDINV_DAG_TREE = 16
SPDINV_DAG_TREE_STEP3 = 32
SPDINV_DAG_SHARE_BC = 64

SPDINV_PROBE_DMMA = 0
SPDINV_PROBE_DFMA = 1
SPDINV_PROBE_FFMA = 2
SPDINV_TIMED_SLICE_GEMM = 0
SPDINV_TIMED_MIXED_DAG = 1
SPDINV_TIMED_FP64_DAG = 2
SPDINV_TIMED_KERNELS = 3

STATUS_NAMES = {0: "SPDINV_OK", -1: "SPDINV_ERR_N", -2: "SPDINV_ERR_LDA", -3: "SPDINV_ERR_NULL",
                -4: "SPDINV_ERR_CUDA", -5: "SPDINV_ERR_TIMEOUT", -6: "SPDINV_ERR_UNSUPPORTED",
                -7: "SPDINV_ERR_WORKSPACE"}


class spdinv_opts(ctypes.Structure):
    _fields_ = [("tile", c_int), ("ctas_per_sm", c_int), ("precision", c_int), ("refine_steps", c_int),
                ("wait_timeout_s", c_double), ("fault_drop_task", c_int), ("residual", c_int),
                ("refine_order", c_int), ("variant", c_int), ("split_segment", c_int),
                ("diag_fp64", c_int)]


# name -> (restype, argtypes); every symbol declared in include/spdinv.h
SIGNATURES = {
    "spdinv_potrf": (c_int, [c_int64, P, c_int64, P, P]),
    "spdinv_trtri": (c_int, [c_int64, P, c_int64, P, P]),
    "spdinv_lauum": (c_int, [c_int64, P, c_int64, P]),
    "spdinv_potri": (c_int, [c_int64, P, c_int64, P, P]),
    "spdinv_potri_ex": (c_int, [c_int64, P, c_int64, ctypes.POINTER(spdinv_opts), P, P]),
    "spdinv_potri_noalloc": (c_int, [c_int64, P, c_int64, P, P]),
    "spdinv_potri_diag": (c_int, [c_int64, P, c_int64, P, P, P]),
    "spdinv_inverse_residual": (c_int, [c_int64, P, c_int64, P, P, c_int, P]),
    "spdinv_potri_batched": (c_int, [c_int, P, P, P, P, P]),
    "spdinv_spotri_batched": (c_int, [c_int, P, P, P, P, P]),
    "spdinv_potri_backward": (c_int, [c_int, c_int64, P, c_int64, c_int64, P, c_int64, c_int64,
                                      P, c_int64, c_int64, P]),
    "spdinv_spotri_backward": (c_int, [c_int, c_int64, P, c_int64, c_int64, P, c_int64, c_int64,
                                       P, c_int64, c_int64, P]),
    "spdinv_batched_tiles": (c_int, [c_int, P]),
    "spdinv_batch_shard": (c_int, [c_int, P, c_int, P, P]),
    "spdinv_plan_emulate": (c_int, [c_int, c_int, c_int, ctypes.c_uint64, c_int, c_int, c_double, c_int, P]),
    "spdinv_plan_check": (c_int, [c_int, c_int, P]),
    "spdinv_slice_tile_order": (c_int, [c_int64, c_int, c_int, P, P, P]),
    "spdinv_plan_emulate_variant": (c_int, [c_int, c_int, c_int, c_int, ctypes.c_uint64, c_int, c_double, c_int, P]),
    "spdinv_workspace_size": (c_int, [c_int64, c_int, ctypes.POINTER(spdinv_opts), P]),
    "spdinv_set_workspace": (c_int, [P, ctypes.c_size_t]),
    "spdinv_mirror_lower": (c_int, [c_int, c_int64, P, c_int64, c_int64, P]),
    "spdinv_smirror_lower": (c_int, [c_int, c_int64, P, c_int64, c_int64, P]),
    "spdinv_dag_critical_path": (c_int, [c_int, c_int, P]),
    "spdinv_dag_task_counts": (c_int, [c_int, P]),
    "spdinv_plan_tasks": (c_int, [c_int64, c_int, c_int, P, c_int64, P, P]),
    "spdinv_plan_simulate": (c_int, [c_int, c_int, c_int, P]),
    "spdinv_set_plan_order": (c_int, [c_int]),
    "spdinv_set_debug_flags": (ctypes.c_uint, [ctypes.c_uint]),
    "spdinv_fp64_peak_probe": (c_int, [c_int, c_int64, c_int, P, P, P]),
    "spdinv_set_kernel_timing": (c_int, [c_int]),
    "spdinv_set_trace": (c_int, [P, c_int64]),
    "spdinv_kernel_time_ms": (c_int, [c_int, P, P, P]),
    "spdinv_status_name": (ctypes.c_char_p, [c_int]),
    "spdinv_last_cuda_error": (ctypes.c_char_p, []),
    "spdinv_kernel_launches": (ctypes.c_uint64, []),
    "spdinv_version": (c_int, []),
}

_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libspdinv.so is missing (%s): run paper_1002_4057_gb300.build.build() "
                               "or __graft_entry__.build() first" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _call(name, *args):
    return getattr(lib(), name)(*args)


def spdinv_potrf(n, dA, lda, d_info, stream):
    return _call("spdinv_potrf", n, dA, lda, d_info, stream)


def spdinv_trtri(n, dA, lda, d_info, stream):
    return _call("spdinv_trtri", n, dA, lda, d_info, stream)


def spdinv_lauum(n, dA, lda, stream):
    return _call("spdinv_lauum", n, dA, lda, stream)


def spdinv_potri(n, dA, lda, d_info, stream):
    return _call("spdinv_potri", n, dA, lda, d_info, stream)


def spdinv_potri_ex(n, dA, lda, opts, d_info, stream):
    return _call("spdinv_potri_ex", n, dA, lda, ctypes.byref(opts) if opts is not None else None, d_info, stream)


def spdinv_inverse_residual(n, dA, lda, dX, dR, residual, stream):
    return _call("spdinv_inverse_residual", n, dA, lda, dX, dR, residual, stream)


def spdinv_potri_diag(n, dA, lda, d_diag, d_info, stream):
    return _call("spdinv_potri_diag", n, dA, lda, d_diag, d_info, stream)


def spdinv_potri_noalloc(n, dA, lda, d_info, stream):
    return _call("spdinv_potri_noalloc", n, dA, lda, d_info, stream)


def spdinv_potri_batched(batch, h_n, d_Aptrs, h_lda, d_info, stream):
    return _call("spdinv_potri_batched", batch, h_n, d_Aptrs, h_lda, d_info, stream)


def spdinv_spotri_batched(batch, h_n, d_Aptrs, h_lda, d_info, stream):
    return _call("spdinv_spotri_batched", batch, h_n, d_Aptrs, h_lda, d_info, stream)


def spdinv_potri_backward(batch, n, dX, ldx, sx, dG, ldg, sg, dGrad, ldgr, sgr, stream):
    return _call("spdinv_potri_backward", batch, n, dX, ldx, sx, dG, ldg, sg, dGrad, ldgr, sgr, stream)


def spdinv_spotri_backward(batch, n, dX, ldx, sx, dG, ldg, sg, dGrad, ldgr, sgr, stream):
    return _call("spdinv_spotri_backward", batch, n, dX, ldx, sx, dG, ldg, sg, dGrad, ldgr, sgr, stream)


def spdinv_batched_tiles(fp32):
    out = (ctypes.c_int * 8)()
    st = _call("spdinv_batched_tiles", int(fp32), ctypes.addressof(out))
    return st, list(out)


def spdinv_batch_shard(sizes, world):
    """(status, owner per matrix, total n^3 per rank) of the split of a batch
    with orders `sizes` across `world` ranks."""
    n = len(sizes)
    hn = (ctypes.c_int * max(n, 1))(*[int(v) for v in sizes])
    owner = (ctypes.c_int * max(n, 1))()
    load = (ctypes.c_double * max(int(world), 1))()
    st = _call("spdinv_batch_shard", n, ctypes.addressof(hn), int(world), ctypes.addressof(owner),
               ctypes.addressof(load))
    return st, list(owner)[:n], list(load)[:max(int(world), 0)]


def spdinv_plan_check(t, steps):
    """(status, [tasks, order differences, critical-path/work difference]) of
    the fast and the exhaustive plan builds."""
    out = (ctypes.c_int64 * 3)()
    st = _call("spdinv_plan_check", int(t), int(steps), ctypes.addressof(out))
    return st, list(out)


def spdinv_slice_tile_order(n, lower, wide=1):
    """(status, bm list, bn list) of the slice GEMM's launch order for order n."""
    cnt = ctypes.c_int(0)
    st = _call("spdinv_slice_tile_order", int(n), int(lower), int(wide), None, None, ctypes.addressof(cnt))
    if st != 0:
        return st, [], []
    bm = (ctypes.c_int * max(cnt.value, 1))()
    bn = (ctypes.c_int * max(cnt.value, 1))()
    st = _call("spdinv_slice_tile_order", int(n), int(lower), int(wide), ctypes.addressof(bm),
               ctypes.addressof(bn), ctypes.addressof(cnt))
    return st, list(bm)[:cnt.value], list(bn)[:cnt.value]


def spdinv_plan_simulate(t, steps, workers):
    """(status, [makespan, work, critical path]) of the plan scheduled on
    `workers` CTAs, in units of one tile product."""
    out = (ctypes.c_double * 3)()
    st = _call("spdinv_plan_simulate", int(t), int(steps), int(workers), ctypes.addressof(out))
    return st, list(out)


def spdinv_workspace_size(n, routine, opts=None):
    """(status, bytes of device workspace) of one call of `routine`."""
    out = ctypes.c_size_t(0)
    st = _call("spdinv_workspace_size", int(n), int(routine), ctypes.byref(opts) if opts is not None else None,
               ctypes.addressof(out))
    return st, out.value


def spdinv_set_workspace(d_ws, nbytes):
    return _call("spdinv_set_workspace", d_ws, int(nbytes))


def spdinv_plan_emulate(t, workers, seed, drop_task=-1, wait_limit_s=5.0, max_delay_us=20, steps=0,
                        skip_wait_task=-1):
    """(status, [completed, tasks, protocol errors, hazards, longest wait in
    us]) of a host emulation of the persistent kernel's scheduling protocol."""
    out = (ctypes.c_int64 * 5)()
    st = _call("spdinv_plan_emulate", int(t), int(steps), int(workers), int(seed), int(drop_task),
               int(skip_wait_task), float(wait_limit_s), int(max_delay_us), ctypes.addressof(out))
    return st, list(out)


def spdinv_plan_emulate_variant(t, variant, workers, seed, split_segment=0, drop_task=-1, wait_limit_s=5.0,
                                max_delay_us=20):
    """(status, [completed, tasks, protocol errors, hazards, longest wait in
    us]) of a host emulation of an execution variant's plan, with the
    kernel's write-after-read protocol."""
    out = (ctypes.c_int64 * 5)()
    st = _call("spdinv_plan_emulate_variant", int(t), int(variant), int(split_segment), int(workers), int(seed),
               int(drop_task), float(wait_limit_s), int(max_delay_us), ctypes.addressof(out))
    return st, list(out)


def spdinv_mirror_lower(batch, n, dA, lda, stride, stream):
    return _call("spdinv_mirror_lower", batch, n, dA, lda, stride, stream)


def spdinv_smirror_lower(batch, n, dA, lda, stride, stream):
    return _call("spdinv_smirror_lower", batch, n, dA, lda, stride, stream)


def spdinv_dag_critical_path(t, flags):
    out = (ctypes.c_int64 * 4)()
    st = _call("spdinv_dag_critical_path", t, flags, ctypes.addressof(out))
    return st, list(out)


def spdinv_dag_task_counts(t):
    out = (ctypes.c_int64 * 12)()
    st = _call("spdinv_dag_task_counts", t, ctypes.addressof(out))
    return st, list(out)


def spdinv_plan_tasks(n, b, steps):
    cnt = ctypes.c_int64(0)
    crit = ctypes.c_double(0)
    st = _call("spdinv_plan_tasks", n, b, steps, None, 0, ctypes.addressof(cnt), ctypes.addressof(crit))
    if st != 0:
        return st, [], 0.0
    buf = (ctypes.c_uint32 * max(cnt.value, 1))()
    st = _call("spdinv_plan_tasks", n, b, steps, ctypes.addressof(buf), cnt.value, ctypes.addressof(cnt),
               ctypes.addressof(crit))
    return st, list(buf)[:cnt.value], crit.value


def spdinv_set_plan_order(order):
    """Sets the ticket order of plans built from now on; returns the previous one."""
    return _call("spdinv_set_plan_order", int(order))


def spdinv_set_debug_flags(flags):
    """Sets the process's debug flags; returns the previous ones."""
    return _call("spdinv_set_debug_flags", int(flags))


def spdinv_fp64_peak_probe(kind, iters, blocks_per_sm, d_sink, stream):
    """(status, flops the queued probe kernel performs)."""
    fl = ctypes.c_double(0)
    st = _call("spdinv_fp64_peak_probe", int(kind), int(iters), int(blocks_per_sm), d_sink,
               ctypes.addressof(fl), stream)
    return st, fl.value


def spdinv_set_trace(d_records, capacity):
    """Sets (or, with d_records None, clears) the per-task trace buffer of the
    current device: capacity records of 48 bytes (spdinv_trace_record)."""
    return _call("spdinv_set_trace", d_records, int(capacity))


def spdinv_set_kernel_timing(on):
    return _call("spdinv_set_kernel_timing", int(on))


def spdinv_kernel_time_ms(which):
    """(status, summed ms, launches, algorithmic flops) of the timed launches
    of one kind since the last query (waits for them to finish)."""
    ms = ctypes.c_double(0)
    cnt = ctypes.c_int(0)
    fl = ctypes.c_double(0)
    st = _call("spdinv_kernel_time_ms", int(which), ctypes.addressof(ms), ctypes.addressof(cnt),
               ctypes.addressof(fl))
    return st, ms.value, cnt.value, fl.value


def spdinv_status_name(status):
    return _call("spdinv_status_name", int(status)).decode()


def spdinv_last_cuda_error():
    return _call("spdinv_last_cuda_error").decode()


def spdinv_kernel_launches():
    return _call("spdinv_kernel_launches")


def spdinv_version():
    return _call("spdinv_version")
