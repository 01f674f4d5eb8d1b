"""Selected inverse diag(A^{-1}) (spdinv_potri_diag): Steps 1 and 2 in full
and Step 3 restricted to the diagonal tiles, against the FP64 CPU oracle's
full inverse.  A is only read."""
import numpy as np
import pytest

import oracle
import spd_inputs as si
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T(gpu):
    from paper_1002_4057_gb300 import torch_api
    return torch_api


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 65, 200, 513, 777])
def test_diag_vs_oracle_and_A_untouched(T, gpu, n):
    import torch
    A, _, _ = si.spectral_spd(n, 1e3, seed=si.SEED_BASE + 40 + n)
    dA = to_dev(A, gpu)
    before = dA.clone()
    info = torch.zeros(1, dtype=torch.int32, device=gpu)
    d = T.inverse_diag(dA, info=info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert torch.equal(dA, before)  # only read
    M, oinfo = oracle.potri(A)
    assert oinfo == 0
    ref = np.diag(M)
    assert np.max(np.abs(d.cpu().numpy() - ref) / np.abs(ref)) <= 1e-11


def test_diag_integer_case_bitwise(T, gpu):
    n = 300
    A, _ = si.bidiag_integer_spd(n, seed=si.SEED_BASE + 41)
    d = T.inverse_diag(to_dev(A, gpu)).cpu().numpy()
    M, _ = oracle.potri(A)
    assert np.array_equal(d, np.diag(M))


def test_diag_equals_full_inverse_diagonal_bitwise(T, gpu):
    """The diagonal tiles run the same chains in the same order as in
    spdinv_potri, so the two diagonals agree bit for bit."""
    import torch
    n = 2000
    A, _, _ = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 42)
    dA = to_dev(A, gpu)
    d = T.inverse_diag(dA)
    W = dA.clone()
    assert int(T.potri_(W).item()) == 0
    torch.cuda.synchronize()
    assert torch.equal(d, torch.diagonal(W))


def test_diag_info_not_positive_definite(T, gpu):
    import torch
    n = 100
    A, _, _ = si.spectral_spd(n, 1e2, seed=si.SEED_BASE + 43)
    A[57, 57] = -1.0
    info = torch.zeros(1, dtype=torch.int32, device=gpu)
    T.inverse_diag(to_dev(A, gpu), info=info)
    _, oinfo = oracle.potri(A)
    assert int(info.item()) == oinfo > 0


def test_diag_argument_errors(T, gpu):
    from paper_1002_4057_gb300 import _lib as L
    assert L.spdinv_potri_diag(-1, 0, 1, 0, 0, 0) == L.SPDINV_ERR_N
    assert L.spdinv_potri_diag(4, 0, 4, 0, 0, 0) == L.SPDINV_ERR_NULL
    assert L.spdinv_potri_diag(0, 0, 1, 0, 0, 0) == L.SPDINV_OK
