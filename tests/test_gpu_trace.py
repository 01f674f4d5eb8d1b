"""Per-task trace of the persistent FP64 kernel (spdinv_set_trace): the
traced run computes the same result bit for bit, records every task of the
plan once at its ticket, and no task finishes before the producers of the
tiles it reads."""
import numpy as np
import pytest

import spd_inputs as si
from gpu_util import lower_np, to_dev

pytestmark = pytest.mark.gpu


def _preds(kind, i, j, t):
    if kind == 0:
        return [(1, j, q) for q in range(j)]
    if kind == 1:
        return [(1, i, q) for q in range(j)] + [(1, j, q) for q in range(j)] + [(0, j, j)]
    if kind == 3:
        return [(0, i, i), (1, i, j), (0, j, j)] + [(3, i, q) for q in range(j + 1, i)] + \
               [(1, q, j) for q in range(j + 1, i)]
    if kind == 5:
        return [(0, i, i), (3, i, j)] + [(3, q, i) for q in range(i + 1, t)] + [(3, q, j) for q in range(i + 1, t)]
    if kind == 4:
        return [(0, i, i)] + [(3, q, i) for q in range(i + 1, t)]
    return []


@pytest.mark.parametrize("n,b", [(300, 32), (777, 32), (640, 64)])
def test_trace_records_every_task_in_dependency_order(gpu, n, b):
    from paper_1002_4057_gb300 import _lib as L
    from paper_1002_4057_gb300 import torch_api as T
    A, _, _ = si.spectral_spd(n, 1e3, seed=n)
    ref = to_dev(A, gpu)
    assert int(T.potri_(ref, tile=b).item()) == 0
    dA = to_dev(A, gpu)
    info, rec = T.traced_potri_(dA, tile=b)
    assert int(info.item()) == 0
    assert np.array_equal(lower_np(dA), lower_np(ref))  # the traced build computes the same
    st, tasks, _ = L.spdinv_plan_tasks(n, b, 0)
    assert st == 0
    rec = rec[:len(tasks)]
    assert np.array_equal(rec["task"], np.array(tasks, dtype=np.uint32))
    assert np.array_equal(rec["ticket"], np.arange(len(tasks)))
    assert np.all(rec["t_end_ns"] >= rec["t_start_ns"]) and np.all(rec["t_start_ns"] > 0)
    assert np.all(rec["t_wait_ns"] <= rec["t_end_ns"] - rec["t_start_ns"])
    t = (n + b - 1) // b
    end = {}
    for r in rec:
        end[(int(r["task"] >> 28), int((r["task"] >> 14) & 0x3FFF), int(r["task"] & 0x3FFF))] = int(r["t_end_ns"])
    for key, e in end.items():
        for p in _preds(*key, t):
            assert e + 2000 >= end[p], (key, p)  # 2 us of timer granularity


def test_trace_buffer_too_small_is_refused(gpu):
    import torch
    from paper_1002_4057_gb300 import _lib as L
    n = 256
    dA = to_dev(np.eye(n), gpu)
    buf = torch.zeros(48 * 4, dtype=torch.uint8, device=gpu)
    assert L.spdinv_set_trace(buf.data_ptr(), 4) == L.SPDINV_OK
    try:
        st = L.spdinv_potri(n, dA.data_ptr(), n, None, torch.cuda.current_stream().cuda_stream)
        assert st == L.SPDINV_ERR_WORKSPACE
    finally:
        assert L.spdinv_set_trace(None, 0) == L.SPDINV_OK
