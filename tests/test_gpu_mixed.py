"""Mixed precision: FP32 bulk tile updates, FP64 diagonal tiles and FP64
residual corrections, against the FP64 oracle.  The error is stated for every
result; the 1e-10 gate applies with the number of correction steps and the
order the conditioning needs (order 2: one step at cond 1e2, two at 1e4;
one step of order 3 at cond 1e2 and of order 4 at cond 1e4)."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
import spd_inputs as si
from gpu_util import full_from_lower, lower_np, to_dev

pytestmark = pytest.mark.gpu

MIXED = 1


def _run(T, A, gpu, steps, tile=64, order=0):
    dA = to_dev(A, gpu)
    info = T.potri_(dA, precision=MIXED, refine_steps=steps, tile=tile, refine_order=order)
    import torch
    torch.cuda.synchronize()
    return dA, int(info.item())


@pytest.mark.parametrize("n", [1, 64, 200, 513, 1000])
@pytest.mark.parametrize("tile", [32, 64])
def test_mixed_error_by_steps(gpu, n, tile):
    from paper_1002_4057_gb300 import torch_api as T
    for cond, steps_needed in ((1e2, 1), (1e4, 2)):
        A, _, _ = si.spectral_spd(n, cond, seed=si.SEED_BASE + 2 + n)
        M, _ = oracle.potri(A)
        ref = oracle.symmetrize_lower(M)
        errs = []
        for steps in range(0, steps_needed + 1):
            dA, info = _run(T, A, gpu, steps, tile)
            assert info == 0
            errs.append(oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref))
        print("n=%d tile=%d cond=%.0e errors by steps: %s" % (n, tile, cond, ["%.2e" % e for e in errs]))
        assert errs[0] <= 1e-3  # the FP32 result itself
        assert errs[-1] <= 1e-10
        if n > 1:
            assert errs[-1] < errs[0]


def test_mixed_integer_case_exact(gpu):
    from paper_1002_4057_gb300 import torch_api as T
    n = 700
    A, s = si.bidiag_integer_spd(n, seed=3)
    for steps, order in ((0, 0), (1, 0), (1, 4), (2, 3)):
        dA, info = _run(T, A, gpu, steps, order=order)
        assert info == 0
        assert np.array_equal(lower_np(dA), np.tril(cf.bidiag_inverse(s)))


@pytest.mark.parametrize("n", [1, 64, 129, 256, 513, 1000, 2300])
def test_mixed_one_step_of_higher_order(gpu, n):
    """One correction of order p: R = I - A X, then X + X R + ... + X R^{p-1}
    with the terms formed as symmetric lower-tile products.  Order 3 at cond
    1e2 and order 4 at cond 1e4 reach the 1e-10 gate in one step; a higher
    order is never worse than order 2 with the same single residual.
    n = 2300 pads to 18 blocks of 128 rows: the slice products' grouped tile
    orders (8 row blocks per group for R, 16 for the lower-tile terms) end in
    a partial group."""
    from paper_1002_4057_gb300 import torch_api as T
    for cond, order in ((1e2, 3), (1e4, 4)):
        A, _, _ = si.spectral_spd(n, cond, seed=si.SEED_BASE + 5 + n)
        M, _ = oracle.potri(A)
        ref = oracle.symmetrize_lower(M)
        errs = {}
        for p in (2, order, 8):
            dA, info = _run(T, A, gpu, 1, order=p)
            assert info == 0
            errs[p] = oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref)
        print("n=%d cond=%.0e one step, error by order: %s" % (n, cond, {k: "%.2e" % v for k, v in errs.items()}))
        assert errs[order] <= 1e-10 and errs[8] <= 1e-10
        assert errs[order] <= max(errs[2], 1e-13)


def test_mixed_two_steps_order3_cond1e6(gpu):
    """cond 1e6: two steps of order 3, against the spectral definition
    Q diag(1/lam) Q^T (the FP64 oracle's own error is ~1e-10 here)."""
    from paper_1002_4057_gb300 import torch_api as T
    n = 700
    A, Q, lam = si.spectral_spd(n, 1e6, seed=si.SEED_BASE + 6)
    ref = (Q / lam) @ Q.T
    dA, info = _run(T, A, gpu, 2, order=3)
    assert info == 0
    err = oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref)
    M, _ = oracle.potri(A)
    e64 = oracle.rel_frobenius(oracle.symmetrize_lower(M), ref)
    print("n=%d cond=1e6 two order-3 steps: error %.2e (FP64 oracle %.2e)" % (n, err, e64))
    assert err <= max(1e-10, 2 * e64)


@pytest.mark.parametrize("n", [1, 64, 513, 1000])
@pytest.mark.parametrize("tile", [32, 64])
@pytest.mark.parametrize("prec", [MIXED, 3])
def test_mixed_fp64_diagonal_tiles(gpu, n, tile, prec):
    """diag_fp64: the DAG's diagonal POTRF/TRTRI in native FP64 (the tile
    converted to FP64 and X_jj rounded back to FP32).  The unrefined result
    is FP32-accurate, one correction of order 4 at cond 1e4 reaches the 1e-10
    gate, and the integer case stays exact."""
    from paper_1002_4057_gb300 import torch_api as T
    A, _, _ = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 7 + n)
    M, _ = oracle.potri(A)
    ref = oracle.symmetrize_lower(M)
    errs = []
    for steps, order in ((0, 0), (1, 4)):
        dA = to_dev(A, gpu)
        info = T.potri_(dA, precision=prec, refine_steps=steps, refine_order=order, tile=tile, diag_fp64=1)
        assert int(info.item()) == 0
        errs.append(oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref))
    print("n=%d tile=%d prec=%d FP64 diagonal tiles: errors %s" % (n, tile, prec, ["%.2e" % e for e in errs]))
    assert errs[0] <= 1e-3 and errs[1] <= 1e-10
    Ai, s_ = si.bidiag_integer_spd(max(n, 2), seed=11)
    dA = to_dev(Ai, gpu)
    info = T.potri_(dA, precision=prec, tile=tile, diag_fp64=1)
    assert int(info.item()) == 0
    assert np.array_equal(lower_np(dA), np.tril(cf.bidiag_inverse(s_)))


def test_mixed_fp64_diagonal_info(gpu):
    from paper_1002_4057_gb300 import torch_api as T
    d = np.ones(300)
    d[150] = -2.0
    dA = to_dev(np.diag(d), gpu)
    info = T.potri_(dA, precision=MIXED, refine_steps=1, diag_fp64=1)
    assert int(info.item()) == 151


def test_mixed_info(gpu):
    from paper_1002_4057_gb300 import torch_api as T
    d = np.ones(300)
    d[150] = -2.0
    dA, info = _run(T, np.diag(d), gpu, 1)
    assert info == 151


@pytest.mark.parametrize("order", [0, 4])
def test_mixed_upper_untouched(gpu, order):
    from paper_1002_4057_gb300 import torch_api as T
    n = 130
    A, _, _ = si.spectral_spd(n, 1e2, seed=8)
    B = A.copy(order="F")
    iu = np.triu_indices(n, 1)
    B[iu] = -3.5
    dA, info = _run(T, B, gpu, 1, order=order)
    assert info == 0
    assert np.all(dA.cpu().numpy()[iu] == -3.5)


@pytest.mark.slow
def test_mixed_full_size_sampled(gpu):
    """n = 16384: sampled columns against the spectral definition
    Q diag(1/lam) Q^T.  At this size the FP32 result's error is ~1e-5 at cond
    1e2 and ~6e-4 at cond 1e4: one order-2 correction reaches ~7e-10 at cond
    1e2 and two reach the 1e-10 gate, as does one of order 3; at cond 1e4 one
    step of order 4 does."""
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    n = 16384
    cols = np.array([0, 7777, 16383])
    for cond, steps, order in ((1e2, 2, 2), (1e2, 1, 3), (1e4, 1, 4)):
        A, Q, lam = si.spectral_spd(n, cond, seed=si.SEED_BASE + 2, device=gpu)
        ref = cf.spectral_inverse_columns(Q.cpu().numpy(), lam, cols)
        del Q
        W = A.clone()
        info = T.potri_(W, precision=MIXED, refine_steps=steps, tile=64, refine_order=order)
        assert int(info.item()) == 0
        Lo = torch.tril(W)
        Xc = (Lo[:, cols] + torch.tril(Lo, -1).t()[:, cols]).cpu().numpy()
        err = np.linalg.norm(Xc - ref) / np.linalg.norm(ref)
        print("n=16384 cond=%.0e steps=%d order=%d sampled error %.2e" % (cond, steps, order, err))
        assert err <= 1e-10
        del A, W, Lo
        torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [1, 31, 127, 128, 129, 300, 1030, 2300])
@pytest.mark.parametrize("residual", [0, 1, 2])
def test_inverse_residual_vs_fp64(gpu, n, residual):
    """R = I - A X against the FP64 CPU product, for an X near A^{-1} (the
    case the correction meets): |R - R_ref| <= 1e-13 |A| |X| elementwise-max.
    n = 1030 and 2300 pad to 10 and 18 blocks of 128 rows, so the tile order
    of the emulated product (groups of 8 row blocks) ends in a partial group."""
    import torch
    from paper_1002_4057_gb300 import _lib as L
    A, _, _ = si.spectral_spd(n, 1e3, seed=900 + n)
    X = np.linalg.inv(A).astype(np.float32).astype(np.float64)  # an FP32-accurate inverse
    X = 0.5 * (X + X.T)
    Rref = np.eye(n) - A @ X
    dA = to_dev(A, gpu)
    dX = torch.from_numpy(np.asfortranarray(X)).to(gpu)
    dR = torch.zeros((n, n), dtype=torch.float64, device=gpu).t()
    st = L.spdinv_inverse_residual(n, dA.data_ptr(), n, dX.data_ptr(), dR.data_ptr(), residual,
                                   torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    R = dR.cpu().numpy()
    scale = np.max(np.abs(A) @ np.abs(X))
    assert np.max(np.abs(R - Rref)) <= 1e-13 * scale, np.max(np.abs(R - Rref)) / scale


@pytest.mark.parametrize("residual", [0, 2])
def test_inverse_residual_exact_integer_case(gpu, residual):
    """Integer A and its exact integer inverse: R must be exactly zero."""
    import torch
    from paper_1002_4057_gb300 import _lib as L
    n = 500
    A, s = si.bidiag_integer_spd(n, seed=5)
    X = cf.bidiag_inverse(s)
    dA = to_dev(A, gpu)
    dX = torch.from_numpy(np.asfortranarray(X)).to(gpu)
    dR = torch.full((n, n), 7.0, dtype=torch.float64, device=gpu).t()
    assert L.spdinv_inverse_residual(n, dA.data_ptr(), n, dX.data_ptr(), dR.data_ptr(), residual,
                                     torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert np.array_equal(dR.cpu().numpy(), np.zeros((n, n)))


@pytest.mark.parametrize("n", [200, 700])
def test_mixed_emulated_matches_native_residual(gpu, n):
    from paper_1002_4057_gb300 import torch_api as T
    A, _, _ = si.spectral_spd(n, 1e4, seed=1200 + n)
    M, _ = oracle.potri(A)
    ref = oracle.symmetrize_lower(M)
    errs = {}
    for residual in (0, 1, 2):
        dA = to_dev(A, gpu)
        info = T.potri_(dA, precision=MIXED, refine_steps=2, tile=64, residual=residual)
        assert int(info.item()) == 0
        errs[residual] = oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref)
    print("n=%d errors emulated(tcgen05) %.2e native %.2e emulated(mma.sync) %.2e" % (n, errs[0], errs[1], errs[2]))
    assert errs[0] <= 1e-10 and errs[1] <= 1e-10 and errs[2] <= 1e-10



def test_torch_wrappers_of_residual_and_noalloc(gpu):
    """torch_api.inverse_residual and potri_noalloc_: the integer case's
    residual is exactly zero, and the no-allocation inversion equals the
    oracle within the FP64 tolerance."""
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    n = 300
    A, s = si.bidiag_integer_spd(n, seed=6)
    X = cf.bidiag_inverse(s)
    R = T.inverse_residual(to_dev(A, gpu), torch.from_numpy(np.asfortranarray(X)).to(gpu))
    assert R.stride() == (1, n)
    assert np.array_equal(R.cpu().numpy(), np.zeros((n, n)))
    A, _, _ = si.spectral_spd(n, 1e3, seed=si.SEED_BASE + 70)
    dA = to_dev(A, gpu)
    assert int(T.potri_noalloc_(dA).item()) == 0
    M, _ = oracle.potri(A)
    assert oracle.rel_frobenius(full_from_lower(lower_np(dA)), oracle.symmetrize_lower(M)) <= 1e-10


# ---- the bulk updates on the tensor cores: 3xTF32 and BF16x3 splits --------
TF32X3, BF16X3 = 3, 2


def _run_prec(T, A, gpu, prec, steps, order=0, tile=64):
    dA = to_dev(A, gpu)
    info = T.potri_(dA, precision=prec, refine_steps=steps, tile=tile, refine_order=order)
    import torch
    torch.cuda.synchronize()
    return dA, int(info.item())


@pytest.mark.parametrize("tile", [32, 64])
@pytest.mark.parametrize("n", [1, 100, 513, 1000])
def test_tf32x3_matches_fp32_accuracy_and_refines(gpu, n, tile):
    """3xTF32 products keep about 21 of FP32's 24 bits per product: the
    unrefined result stays within a small factor of the FP32 one (both
    against the oracle), and one order-4 correction reaches 1e-10 at cond
    1e4, as with FP32 updates."""
    from paper_1002_4057_gb300 import torch_api as T
    A, _, _ = si.spectral_spd(n, 1e4, seed=si.SEED_BASE + 11 + n)
    M, _ = oracle.potri(A)
    ref = oracle.symmetrize_lower(M)
    d32, i32 = _run_prec(T, A, gpu, MIXED, 0, tile=tile)
    dtc, itc = _run_prec(T, A, gpu, TF32X3, 0, tile=tile)
    assert i32 == 0 and itc == 0
    e32 = oracle.rel_frobenius(full_from_lower(lower_np(d32)), ref)
    etc = oracle.rel_frobenius(full_from_lower(lower_np(dtc)), ref)
    print("n=%d tile=%d cond 1e4 unrefined: FP32 %.2e, 3xTF32 %.2e" % (n, tile, e32, etc))
    assert etc <= max(16 * e32, 1e-12) and etc <= 1e-2
    dA, info = _run_prec(T, A, gpu, TF32X3, 1, order=4, tile=tile)
    assert info == 0
    e = oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref)
    print("  3xTF32 + one order-4 step: %.2e" % e)
    assert e <= 1e-10


@pytest.mark.parametrize("n", [1, 100, 513, 1000])
def test_bf16x3_error_and_refinement(gpu, n):
    """BF16x3 keeps about 16 bits per product: the unrefined result's error is
    larger (stated), and at cond 1e2 two corrections of order 3 reach 1e-10."""
    from paper_1002_4057_gb300 import torch_api as T
    A, _, _ = si.spectral_spd(n, 1e2, seed=si.SEED_BASE + 13 + n)
    M, _ = oracle.potri(A)
    ref = oracle.symmetrize_lower(M)
    d0, i0 = _run_prec(T, A, gpu, BF16X3, 0)
    assert i0 == 0
    e0 = oracle.rel_frobenius(full_from_lower(lower_np(d0)), ref)
    dA, info = _run_prec(T, A, gpu, BF16X3, 2, order=3)
    assert info == 0
    e2 = oracle.rel_frobenius(full_from_lower(lower_np(dA)), ref)
    print("n=%d cond 1e2: BF16x3 unrefined %.2e, two order-3 steps %.2e" % (n, e0, e2))
    assert e0 <= 5e-2
    assert e2 <= 1e-10


@pytest.mark.parametrize("prec", [TF32X3, BF16X3])
def test_split_precisions_exact_on_integer_case(gpu, prec):
    """Entries of the integer test matrix are small integers: their high
    parts are exact and the low parts zero, so every product is exact and the
    result bitwise."""
    from paper_1002_4057_gb300 import torch_api as T
    n = 700
    A, s = si.bidiag_integer_spd(n, seed=3)
    for steps, order in ((0, 0), (1, 4)):
        dA, info = _run_prec(T, A, gpu, prec, steps, order=order)
        assert info == 0
        assert np.array_equal(lower_np(dA), np.tril(cf.bidiag_inverse(s)))


@pytest.mark.parametrize("prec", [TF32X3, BF16X3])
def test_split_precisions_report_the_failing_column(gpu, prec):
    from paper_1002_4057_gb300 import torch_api as T
    n = 300
    A, _, _ = si.spectral_spd(n, 1e2, seed=5)
    A[150, 150] = -1.0
    _, oinfo = oracle.potri(A)
    _, info = _run_prec(T, A, gpu, prec, 1)
    assert oinfo > 0 and info == oinfo
