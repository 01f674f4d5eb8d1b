"""The execution variants of the FP64 plan (the study of Sec. 3 on the GPU:
loop order UUU, renaming under a memory budget with C in B's slots, no
renaming at all, and Step-3 chains split into segments) against the FP64 CPU
oracle, through the C-ABI.

Each variant changes where tiles are stored, which tasks wait for which, and
(UUU, split chains) the order in which a chain's products are added, so the
results agree with the oracle by tolerance -- relative Frobenius error
<= 1e-10 and LAPACK ratio <= 10 at cond <= 1e4, as for the default plan -- and,
on the integer test matrix whose every intermediate is a small integer, bit
for bit."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
import spd_inputs as si
from gpu_util import full_from_lower, lower_np, to_dev

pytestmark = pytest.mark.gpu

UUU, SHARE, INPLACE, SPLIT = 1, 2, 4, 8
VARIANTS = [(UUU, 0), (SHARE, 0), (INPLACE, 0), (UUU | SHARE, 0), (UUU | INPLACE, 0), (SPLIT, 1), (SPLIT, 3),
            (SPLIT | UUU, 2)]
IDS = ["uuu", "share_bc", "inplace", "uuu_share", "uuu_inplace", "split1", "split3", "split2_uuu"]


@pytest.fixture(scope="module")
def T(gpu):
    from paper_1002_4057_gb300 import torch_api
    return torch_api


def _sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("var,seg", VARIANTS, ids=IDS)
@pytest.mark.parametrize("n,b", [(1, 32), (33, 32), (200, 32), (513, 32), (777, 64), (1000, 32)])
def test_variant_vs_oracle(T, gpu, var, seg, n, b):
    A, _, _ = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 31 * n + var)
    dA = to_dev(A, gpu, lda=n + 3)
    upper = np.triu(A, 1)
    info = T.potri_(dA, tile=b, variant=var, split_segment=seg)
    _sync()
    assert int(info.item()) == 0
    got = dA.cpu().numpy()
    assert np.array_equal(np.triu(got, 1), upper)  # the strictly upper part is never touched
    X = full_from_lower(np.tril(got))
    M, oinfo = oracle.potri(A)
    assert oinfo == 0
    assert oracle.rel_frobenius(X, oracle.symmetrize_lower(M)) <= 1e-10
    assert oracle.lapack_ratio(A, X) <= 10


@pytest.mark.parametrize("var,seg", VARIANTS, ids=IDS)
@pytest.mark.parametrize("n", [64, 300, 1000])
def test_variant_integer_bitwise(T, gpu, var, seg, n):
    A, s = si.bidiag_integer_spd(n, seed=n + 29)
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA, tile=32, variant=var, split_segment=seg).item()) == 0
    assert np.array_equal(lower_np(dA), np.tril(cf.bidiag_inverse(s)))


@pytest.mark.parametrize("var,seg", VARIANTS, ids=IDS)
def test_variant_tridiag_closed_form(T, gpu, var, seg):
    n = 512
    dA = to_dev(si.tridiag(n), gpu)
    assert int(T.potri_(dA, tile=32, variant=var, split_segment=seg).item()) == 0
    assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), cf.tridiag_inverse(n)) <= 1e-10


@pytest.mark.parametrize("var,seg", VARIANTS, ids=IDS)
def test_variant_result_does_not_depend_on_the_grid(T, gpu, var, seg):
    n = 700
    A, _, _ = si.spectral_spd(n, 1e3, seed=77)
    outs = []
    for per in (1, 2, 0):
        dA = to_dev(A, gpu)
        assert int(T.potri_(dA, tile=32, ctas_per_sm=per, variant=var, split_segment=seg).item()) == 0
        outs.append(lower_np(dA))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("var,seg", [(UUU, 0), (SHARE, 0), (INPLACE, 0), (SPLIT, 2)],
                         ids=["uuu", "share_bc", "inplace", "split2"])
def test_variant_reports_the_first_failing_column(T, gpu, var, seg):
    n = 300
    A, _, _ = si.spectral_spd(n, 1e2, seed=5)
    A[150, 150] = -1.0  # the leading minor of order 151 is not positive definite
    M, oinfo = oracle.potri(A)
    dA = to_dev(A, gpu)
    info = int(T.potri_(dA, tile=32, variant=var, split_segment=seg).item())
    assert oinfo > 0 and info == oinfo


def test_variant_options_are_checked(T, gpu):
    import torch
    from paper_1002_4057_gb300 import _lib as L
    dA = to_dev(np.eye(64), gpu)
    s = torch.cuda.current_stream().cuda_stream
    info = torch.zeros(1, dtype=torch.int32, device=gpu)
    for var in (16, SPLIT | SHARE, SPLIT | INPLACE):
        o = L.spdinv_opts(32, 0, 0, 0, 0.0, -1, 0, 0, var, 0)
        assert L.spdinv_potri_ex(64, dA.data_ptr(), 64, o, info.data_ptr(), s) == L.SPDINV_ERR_UNSUPPORTED
    o = L.spdinv_opts(32, 0, 1, 0, 0.0, -1, 0, 0, UUU, 0)  # variants are FP64 only
    assert L.spdinv_potri_ex(64, dA.data_ptr(), 64, o, info.data_ptr(), s) == L.SPDINV_ERR_UNSUPPORTED
