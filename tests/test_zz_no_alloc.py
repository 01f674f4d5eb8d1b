"""spdinv_potri_noalloc: the inversion for callers that cannot allocate
device memory (a host application that owns all device memory, loops where
an allocation's device-wide synchronisation would stall other streams).  Its
scratch is a fixed array inside the library.

It is checked through the C-ABI against spdinv_potri (tile 32) on two calls
in a row, within the FP64 parity tolerance of the other tests (relative
Frobenius error 1e-10); each tile's update chain runs in the same order on
both paths, so the two results are also equal bit for bit.  The second call reuses the array the first one left
behind, and must neither allocate device memory nor see stale state.
This file is collected last, so a failure here stops a -x run only after
every other test has run."""
import numpy as np
import pytest

import spd_inputs as si
from gpu_util import full_from_lower, lower_np, to_dev

pytestmark = pytest.mark.gpu


def _rel(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def test_noalloc_matches_potri_on_two_calls_in_a_row(gpu):
    import torch
    from paper_1002_4057_gb300 import _lib as L
    from paper_1002_4057_gb300 import torch_api as T

    stream = torch.cuda.current_stream()
    cases = [(1000, 1e3, 11), (333, 1e4, 12)]  # the second is smaller: stale tiles must not leak in
    prepared = []
    for n, cond, seed in cases:
        A, _, _ = si.spectral_spd(n, cond, seed=seed)
        ref = to_dev(A, gpu)
        assert int(T.potri_(ref, tile=32).item()) == 0
        prepared.append((n, to_dev(A, gpu), full_from_lower(lower_np(ref)),
                         torch.full((1,), 99, dtype=torch.int32, device=gpu)))
    torch.cuda.synchronize()

    for call, (n, dA, ref_full, info) in enumerate(prepared):
        free_before = torch.cuda.mem_get_info(gpu)[0]
        st = L.spdinv_potri_noalloc(n, dA.data_ptr(), dA.stride(1), info.data_ptr(), stream.cuda_stream)
        assert st == L.SPDINV_OK, L.STATUS_NAMES.get(st, st)
        torch.cuda.synchronize()
        if call > 0:  # after the one-time set-up, a call allocates nothing
            assert torch.cuda.mem_get_info(gpu)[0] == free_before
        assert int(info.item()) == 0
        got = full_from_lower(lower_np(dA))
        assert _rel(got, ref_full) <= 1e-10
        assert np.array_equal(got, ref_full)


def test_noalloc_rejects_sizes_beyond_its_maximum(gpu):
    import torch
    from paper_1002_4057_gb300 import _lib as L
    n = L.SPDINV_NOALLOC_MAX_N + 1
    dA = torch.zeros((n, n), dtype=torch.float64, device=gpu).t()
    st = L.spdinv_potri_noalloc(n, dA.data_ptr(), n, None, torch.cuda.current_stream().cuda_stream)
    assert st == L.SPDINV_ERR_N
