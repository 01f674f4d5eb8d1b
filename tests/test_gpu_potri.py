"""Parity of the CUDA FP64 path (through the C-ABI) with the FP64 CPU oracle.

Tolerances (the FP64 gates of the inversion): LAPACK ratio
||I - A X||_1 / (n ||A||_1 ||X||_1 eps) <= 10 and relative Frobenius error
vs the oracle <= 1e-10 for cond(A) <= 1e4; the integer case is bitwise."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
import spd_inputs as si
from gpu_util import full_from_lower, lower_np, to_dev

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 32, 33, 64, 65, 100, 200, 512, 513, 777]


@pytest.fixture(scope="module")
def T(gpu):
    from paper_1002_4057_gb300 import torch_api
    return torch_api


def _sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("b", [32, 64])
@pytest.mark.parametrize("n", SIZES)
def test_potri_vs_oracle(T, gpu, n, b):
    A, _, _ = si.spectral_spd(n, 1e3, seed=si.SEED_BASE + n)
    dA = to_dev(A, gpu)
    info = T.potri_(dA, tile=b)
    _sync()
    assert int(info.item()) == 0
    X = full_from_lower(lower_np(dA))
    M, oinfo = oracle.potri(A)
    assert oinfo == 0
    assert oracle.rel_frobenius(X, oracle.symmetrize_lower(M)) <= 1e-10
    assert oracle.lapack_ratio(A, X) <= 10


@pytest.mark.parametrize("cond", [1e2, 1e4])
def test_potri_config_n512_tile64(T, gpu, cond):
    n = 512
    A, _, _ = si.spectral_spd(n, cond, seed=si.SEED_BASE)
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA, tile=64).item()) == 0
    X = full_from_lower(lower_np(dA))
    M, _ = oracle.potri(A)
    assert oracle.rel_frobenius(X, oracle.symmetrize_lower(M)) <= 1e-10
    assert oracle.lapack_ratio(A, X) <= 10


@pytest.mark.parametrize("b", [32, 64])
def test_potri_tridiag_closed_form(T, gpu, b):
    n = 512
    dA = to_dev(si.tridiag(n), gpu)
    assert int(T.potri_(dA, tile=b).item()) == 0
    X = full_from_lower(lower_np(dA))
    # cond(T) ~ 1.07e5 at n = 512
    assert oracle.rel_frobenius(X, cf.tridiag_inverse(n)) <= 1e-10


@pytest.mark.parametrize("b", [32, 64])
@pytest.mark.parametrize("n", [1, 5, 64, 300, 1000, 2049])
def test_potri_integer_bitwise(T, gpu, n, b):
    A, s = si.bidiag_integer_spd(n, seed=n + 17)
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA, tile=b).item()) == 0
    assert np.array_equal(lower_np(dA), np.tril(cf.bidiag_inverse(s)))


@pytest.mark.parametrize("n", [1, 70, 300, 1000])
def test_steps_separately(T, gpu, n):
    from paper_1002_4057_gb300 import _lib as L
    import torch
    A, _, _ = si.spectral_spd(n, 1e3, seed=7 + n)
    Lr, _ = oracle.potrf(A)
    Xr, _ = oracle.trtri(Lr)
    Mr = oracle.lauum(Xr)
    # potrf
    dA = to_dev(A, gpu)
    assert int(T.potrf_(dA).item()) == 0
    _sync()
    Lg = lower_np(dA)
    assert np.linalg.norm(Lg - np.tril(Lr)) <= 1e-12 * np.linalg.norm(np.tril(Lr))
    # trtri on the oracle's factor
    dL = to_dev(np.tril(Lr), gpu)
    assert int(T.trtri_(dL).item()) == 0
    _sync()
    assert np.linalg.norm(lower_np(dL) - np.tril(Xr)) <= 1e-11 * np.linalg.norm(np.tril(Xr))
    # lauum on the oracle's inverse factor
    dX = to_dev(np.tril(Xr), gpu)
    T.lauum_(dX)
    _sync()
    assert np.linalg.norm(lower_np(dX) - np.tril(Mr)) <= 1e-12 * np.linalg.norm(np.tril(Mr))


def test_trtri_then_lauum_is_lapack_potri_on_a_factor(T, gpu):
    n = 450
    A, _, _ = si.spectral_spd(n, 1e3, seed=31)
    Lr, _ = oracle.potrf(A)
    dA = to_dev(np.tril(Lr), gpu)
    T.trtri_(dA)
    T.lauum_(dA)
    _sync()
    M, _ = oracle.potri(A)
    assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), oracle.symmetrize_lower(M)) <= 1e-10


def test_upper_triangle_untouched_and_lda(T, gpu):
    import torch
    n, lda = 257, 300
    A, _, _ = si.spectral_spd(n, 1e2, seed=3)
    B = A.copy(order="F")
    iu = np.triu_indices(n, 1)
    B[iu] = 7.25
    dA = to_dev(B, gpu, lda=lda)
    assert int(T.potri_(dA).item()) == 0
    _sync()
    out = dA.cpu().numpy()
    assert np.all(out[iu] == 7.25)
    # padding rows between n and lda are never written
    store = dA.as_strided((n * lda,), (1,)).cpu().numpy().reshape(n, lda)
    assert np.all(np.isnan(store[:, n:]))
    M, _ = oracle.potri(A)
    assert oracle.rel_frobenius(full_from_lower(np.tril(out)), oracle.symmetrize_lower(M)) <= 1e-10


@pytest.mark.parametrize("b", [32, 64])
@pytest.mark.parametrize("bad_col", [0, 40, 129, 199])
def test_info_not_positive_definite(T, gpu, b, bad_col):
    n = 200
    d = np.linspace(1.0, 2.0, n)
    d[bad_col] = -1.0
    A = np.diag(d)
    _, oinfo = oracle.potri(A)
    assert oinfo == bad_col + 1
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA, tile=b).item()) == bad_col + 1
    dA = to_dev(A, gpu)
    assert int(T.potrf_(dA).item()) == bad_col + 1


def test_info_nan(T, gpu):
    A, _, _ = si.spectral_spd(100, 1e2, seed=4)
    A[50, 50] = np.nan
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA).item()) == 51


def test_trtri_zero_diagonal_leaves_A(T, gpu):
    n = 150
    Lm = np.tril(np.ones((n, n))) + np.eye(n)
    Lm[77, 77] = 0.0
    dA = to_dev(Lm, gpu)
    assert int(T.trtri_(dA).item()) == 78
    _sync()
    assert np.array_equal(dA.cpu().numpy(), Lm)


def test_n0(T, gpu):
    import torch
    dA = torch.zeros((0, 0), dtype=torch.float64, device=gpu)
    info = torch.full((1,), 5, dtype=torch.int32, device=gpu)
    T.potri_(dA, info=info)
    assert int(info.item()) == 0


@pytest.mark.parametrize("b", [32, 64])
def test_bitwise_determinism_across_grids(T, gpu, b):
    n = 900
    A, _, _ = si.spectral_spd(n, 1e3, seed=77)
    outs = []
    for per in (1, 2, 0):
        dA = to_dev(A, gpu)
        assert int(T.potri_(dA, tile=b, ctas_per_sm=per).item()) == 0
        outs.append(lower_np(dA))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_wait_limit_returns_timeout_and_context_survives(T, gpu):
    from paper_1002_4057_gb300 import _lib as L
    n = 640
    A, _, _ = si.spectral_spd(n, 1e2, seed=5)
    dA = to_dev(A, gpu)
    # the task with ticket 0 never signals: its consumers give up after 0.2 s
    info = T.potri_(dA, tile=64, wait_timeout_s=0.2, fault_drop_task=0)
    _sync()
    assert int(info.item()) == L.SPDINV_ERR_TIMEOUT
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA, tile=64).item()) == 0
    M, _ = oracle.potri(A)
    assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), oracle.symmetrize_lower(M)) <= 1e-10


def test_full_size_n4096_sampled(T, gpu):
    """n = 4096 (tile sweep workload): sampled columns of the exact inverse
    Q diag(1/lam) Q^T, and the O(n^2) probe ||A (X v) - v|| / ||v||."""
    import torch
    n = 4096
    A, Q, lam = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 1, device=gpu)
    Qh = Q.cpu().numpy()
    Ah = A.cpu().numpy()
    cols = np.array([0, 1, 63, 64, 2047, 4095])
    ref = cf.spectral_inverse_columns(Qh, lam, cols)
    for b in (32, 64):
        dA = A.clone()
        assert int(T.potri_(dA, tile=b).item()) == 0
        X = full_from_lower(dA.cpu().numpy())
        err = np.linalg.norm(X[:, cols] - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, err
        v = np.random.default_rng(1).standard_normal(n)
        assert np.linalg.norm(Ah @ (X @ v) - v) / np.linalg.norm(v) <= 1e4 * n * 2.0 ** -53 * 10


@pytest.mark.slow
def test_full_size_n16384_sampled(T, gpu):
    """n = 16384, tiles 32 (the benchmarked configuration) and 64: integer
    case checked bitwise on whole sampled rows, spectral case on sampled
    columns."""
    import torch
    n = 16384
    # integer bidiagonal: bitwise
    A, s = si.bidiag_integer_spd(n, seed=9)
    A0 = torch.from_numpy(A).to(gpu)
    del A
    rows = np.array([0, 1, 4095, 8191, 8192, 16383])
    r, c = np.meshgrid(rows, np.arange(n), indexing="ij")
    exp = cf.bidiag_inverse_entries(s, r, c)
    mask = c <= r
    for b in (32, 64):
        dA = A0.clone()
        assert int(T.potri_(dA, tile=b).item()) == 0
        got = dA[rows, :].cpu().numpy()
        assert np.array_equal(got[mask], exp[mask]), b
        del dA
    del A0
    torch.cuda.empty_cache()
    # spectral, cond 1e4
    A0, Q, lam = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 1, device=gpu)
    cols = np.array([0, 5000, 16383])
    ref = cf.spectral_inverse_columns(Q.cpu().numpy(), lam, cols)
    del Q
    for b in (32, 64):
        A = A0.clone()
        assert int(T.potri_(A, tile=b).item()) == 0
        Lo = torch.tril(A)
        Xc = (Lo[:, cols] + torch.tril(Lo, -1).t()[:, cols]).cpu().numpy()
        err = np.linalg.norm(Xc - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (b, err)
        del A, Lo


def test_caller_workspace_and_graph_capture(T, gpu):
    """spdinv_set_workspace: the FP64 and the mixed inversion run in a
    caller's buffer of spdinv_workspace_size bytes and match the oracle; a
    buffer 256 bytes too small is refused before any work; with the plan
    built by a first call, a call in the caller's buffer is captured in a
    CUDA graph and replayed."""
    import torch
    n = 300
    A, _, _ = si.spectral_spd(n, 1e2, seed=si.SEED_BASE + 50)
    M, oinfo = oracle.potri(A)
    assert oinfo == 0
    ref = oracle.symmetrize_lower(M)
    need = T.workspace_size(n)
    need_mixed = T.workspace_size(n, precision=1, refine_steps=1, refine_order=3)
    buf = torch.empty(max(need, need_mixed), dtype=torch.uint8, device=gpu)
    T.set_workspace(buf)
    try:
        dA = to_dev(A, gpu)
        assert int(T.potri_(dA).item()) == 0
        assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref) <= 1e-10
        dA = to_dev(A, gpu)
        assert int(T.potri_(dA, precision=1, refine_steps=1, refine_order=3).item()) == 0
        assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref) <= 1e-10

        T.set_workspace(buf[:need - 256])
        with pytest.raises(T.SpdinvError, match="SPDINV_ERR_WORKSPACE"):
            T.potri_(to_dev(A, gpu))

        T.set_workspace(buf[:need])
        dA = to_dev(A, gpu)
        orig = dA.clone()
        info = torch.zeros(1, dtype=torch.int32, device=gpu)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            T.potri_(dA, info=info, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            T.potri_(dA, info=info)
        for _ in range(2):
            dA.copy_(orig)
            info.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            assert int(info.item()) == 0
            assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref) <= 1e-10
    finally:
        T.set_workspace(None)


@pytest.mark.parametrize("n", [1, 33, 100, 257])
def test_poisoned_stores_are_never_read_unwritten(T, gpu, n):
    """SPDINV_DEBUG_POISON: B, C and D start as NaN in every call, so a tile
    read before its producer wrote it would make the result NaN.  The
    pipelined inversion (tiles 32 and 64), the three steps one after the
    other and the selected inverse still match the oracle."""
    from paper_1002_4057_gb300 import _lib as L
    A, _, _ = si.spectral_spd(n, 1e3, seed=si.SEED_BASE + 60 + n)
    M, oinfo = oracle.potri(A)
    assert oinfo == 0
    ref = oracle.symmetrize_lower(M)
    old = L.spdinv_set_debug_flags(L.SPDINV_DEBUG_POISON)
    try:
        for b in (32, 64):
            dA = to_dev(A, gpu)
            assert int(T.potri_(dA, tile=b).item()) == 0
            assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref) <= 1e-10
        dA = to_dev(A, gpu)
        assert int(T.potrf_(dA).item()) == 0
        assert int(T.trtri_(dA).item()) == 0
        T.lauum_(dA)
        assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref) <= 1e-10
        d = T.inverse_diag(to_dev(A, gpu)).cpu().numpy()
        assert np.max(np.abs(d - np.diag(ref)) / np.abs(np.diag(ref))) <= 1e-10
    finally:
        L.spdinv_set_debug_flags(old)


@pytest.mark.parametrize("n", [1, 100, 128, 129, 300, 513, 1000])
def test_potri_tile128_vs_oracle(T, gpu, n):
    """Tile 128 (256-thread CTAs, operands streamed in 32-deep slabs through
    2-D tensor maps) against the oracle, at the FP64 gates."""
    A, _, _ = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 3 * n)
    dA = to_dev(A, gpu, lda=n + 1)
    upper = np.triu(A, 1)
    info = T.potri_(dA, tile=128)
    _sync()
    assert int(info.item()) == 0
    got = dA.cpu().numpy()
    assert np.array_equal(np.triu(got, 1), upper)
    X = full_from_lower(np.tril(got))
    M, _ = oracle.potri(A)
    assert oracle.rel_frobenius(X, oracle.symmetrize_lower(M)) <= 1e-10
    assert oracle.lapack_ratio(A, X) <= 10


@pytest.mark.parametrize("n", [5, 300, 1000])
def test_potri_tile128_integer_bitwise_and_info(T, gpu, n):
    A, s = si.bidiag_integer_spd(n, seed=n + 91)
    dA = to_dev(A, gpu)
    assert int(T.potri_(dA, tile=128).item()) == 0
    assert np.array_equal(lower_np(dA), np.tril(cf.bidiag_inverse(s)))
    B, _, _ = si.spectral_spd(n, 1e2, seed=n)
    B[n // 2, n // 2] = -1.0
    _, oinfo = oracle.potri(B)
    assert int(T.potri_(to_dev(B, gpu), tile=128).item()) == oinfo > 0


def test_potri_tile128_only_for_the_whole_inversion(T, gpu):
    import torch
    from paper_1002_4057_gb300 import _lib as L
    o = L.spdinv_opts(128, 0, 0, 0, 0.0, -1, 0, 0, L.SPDINV_VARIANT_UUU, 0)
    dA = to_dev(np.eye(256), gpu)
    assert L.spdinv_potri_ex(256, dA.data_ptr(), 256, o, None, torch.cuda.current_stream().cuda_stream) == \
        L.SPDINV_ERR_UNSUPPORTED
