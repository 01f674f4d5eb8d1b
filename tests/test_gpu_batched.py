"""Batched inversion of uneven sizes in one launch (FP64 and FP32) against
the FP64 oracle per matrix; CUDA-graph capture; autotuner table."""
import numpy as np
import pytest

import oracle
import spd_inputs as si
from gpu_util import full_from_lower, to_dev

pytestmark = pytest.mark.gpu


def _mats(sizes, dtype, gpu, seed):
    import torch
    hs = si.wishart_batch(sizes, 0.1, seed)
    ds = [to_dev(A, gpu).to(dtype) if dtype != torch.float64 else to_dev(A, gpu) for A in hs]
    # .to(dtype) keeps strides (column-major)
    return hs, ds


def _check(hs, ds, tol):
    worst = 0.0
    for A, d in zip(hs, ds):
        M, info = oracle.potri(A)
        assert info == 0
        X = full_from_lower(np.tril(d.double().cpu().numpy()))
        worst = max(worst, oracle.rel_frobenius(X, oracle.symmetrize_lower(M)))
    print("batched: worst relative Frobenius error vs the oracle %.3e (tolerance %.1e)" % (worst, tol))
    assert worst <= tol, worst
    return worst


# FP32: the inputs are the FP64 matrices rounded to FP32 (cond <= ~41 for
# B B^T/n + 0.1 I), so the error against the FP64 oracle is of order
# cond * 2^-24 * sqrt(n); the worst measured over these tests on a GB300 is
# 1.42e-6, and the tolerance is about 4x that.
F32_TOL = 6e-6


@pytest.mark.parametrize("dtype_name,tol", [("float64", 1e-10), ("float32", F32_TOL)])
def test_batched_uneven_vs_oracle(gpu, dtype_name, tol):
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    dtype = getattr(torch, dtype_name)
    sizes = si.batch_sizes(300, 1, 300, seed=5)
    sizes[:6] = [1, 2, 16, 17, 256, 300]
    hs, ds = _mats(sizes, dtype, gpu, 21)
    info = T.potri_batched_(ds)
    torch.cuda.synchronize()
    assert int(info.abs().sum().item()) == 0
    _check(hs, ds, tol)


def test_batched_integer_bitwise(gpu):
    import torch
    from oracle import closed_forms as cf
    from paper_1002_4057_gb300 import torch_api as T
    sizes = [1, 5, 16, 31, 33, 64, 100, 129, 256, 257]
    hs, ss, ds = [], [], []
    for k, n in enumerate(sizes):
        A, s = si.bidiag_integer_spd(n, seed=40 + k)
        hs.append(A); ss.append(s); ds.append(to_dev(A, gpu))
    T.potri_batched_(ds)
    torch.cuda.synchronize()
    for s, d in zip(ss, ds):
        assert np.array_equal(np.tril(d.cpu().numpy()), np.tril(cf.bidiag_inverse(s)))


def test_batched_equals_single_matrix_call(gpu):
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    sizes = [40, 200]
    hs, ds = _mats(sizes, torch.float64, gpu, 3)
    T.potri_batched_(ds)
    for A, d in zip(hs, ds):
        e = to_dev(A, gpu)
        T.potri_(e)
        torch.cuda.synchronize()
        X1 = full_from_lower(np.tril(d.cpu().numpy()))
        X2 = full_from_lower(np.tril(e.cpu().numpy()))
        assert oracle.rel_frobenius(X1, X2) <= 1e-12


def test_batched_info_per_matrix(gpu):
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    good = si.wishart_spd(50, 0.1, seed=1)
    bad = np.diag(np.r_[np.ones(70), -1.0, np.ones(29)])
    ds = [to_dev(good, gpu), to_dev(bad, gpu), to_dev(good[:10, :10], gpu)]
    info = T.potri_batched_(ds)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 71, 0]


def test_batched_cuda_graph_replay(gpu):
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    sizes = si.batch_sizes(200, 16, 256, seed=9)
    hs, ds = _mats(sizes, torch.float64, gpu, 33)
    originals = [d.clone() for d in ds]
    pb = T.PreparedBatch(ds)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pb.run(s)  # first call: plan built and uploaded outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for d, o in zip(ds, originals):
        d.copy_(o)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pb.run()
    for rep in range(2):
        for d, o in zip(ds, originals):
            d.copy_(o)
        g.replay()
        torch.cuda.synchronize()
        assert int(pb.info.abs().sum().item()) == 0
        _check(hs[:40], ds[:40], 1e-10)


def test_autotuner_table(gpu):
    from paper_1002_4057_gb300 import _lib as L
    for fp32 in (0, 1):
        st, tiles = L.spdinv_batched_tiles(fp32)
        assert st == 0
        allowed = {16, 32} if fp32 == 0 else {16, 32, 64}
        assert all(t in allowed for t in tiles), tiles



@pytest.mark.parametrize("dtype_name,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_sharded_batch_matches_whole_batch(gpu, dtype_name, tol):
    """The multi-GPU path on one GPU, rank after rank: spdinv_batch_shard
    splits the batch for two ranks, each share goes through its own batched
    call, and every matrix matches the whole-batch call (a share may get a
    different tile plan, so the comparison is by tolerance) and the oracle."""
    import torch
    from paper_1002_4057_gb300 import _lib as L
    from paper_1002_4057_gb300 import torch_api as T
    dtype = getattr(torch, dtype_name)
    sizes = si.batch_sizes(120, 16, 256, seed=17)
    hs, whole = _mats(sizes, dtype, gpu, 23)
    assert int(T.potri_batched_(whole).abs().sum().item()) == 0
    st, owner, load = L.spdinv_batch_shard([int(v) for v in sizes], 2)
    assert st == 0 and sorted(set(owner)) == [0, 1]
    got = [None] * len(sizes)
    for rank in (0, 1):
        mine = [k for k in range(len(sizes)) if owner[k] == rank]
        share = [to_dev(hs[k], gpu).to(dtype) for k in mine]  # .to keeps the column-major strides
        assert int(T.potri_batched_(share).abs().sum().item()) == 0
        for d, k in zip(share, mine):
            got[k] = d
    torch.cuda.synchronize()
    for k in range(len(sizes)):
        a = full_from_lower(np.tril(got[k].double().cpu().numpy()))
        b = full_from_lower(np.tril(whole[k].double().cpu().numpy()))
        assert oracle.rel_frobenius(a, b) <= tol, (k, sizes[k])
    _check(hs, got, 1e-10 if dtype == torch.float64 else F32_TOL)

@pytest.mark.slow
def test_batched_config_4096_sampled(gpu):
    """The 4096-matrix workload (n ~ U{16..256}, A = B B^T/n + 0.1 I): every
    matrix checked by the O(n^2) probe ||A (X v) - v|| / ||v||, a sample by
    the oracle."""
    import torch
    from paper_1002_4057_gb300 import torch_api as T
    sizes = si.batch_sizes(4096, 16, 256, seed=si.SEED_BASE + 3)
    hs = si.wishart_batch(sizes, 0.1, si.SEED_BASE + 3)
    for dtype, tol, ptol in ((torch.float64, 1e-10, 1e-11), (torch.float32, F32_TOL, 1e-3)):
        ds = [to_dev(A, gpu).to(dtype) for A in hs]
        info = T.potri_batched_(ds)
        torch.cuda.synchronize()
        assert int(info.abs().sum().item()) == 0
        rng = np.random.default_rng(0)
        for A, d in zip(hs, ds):
            X = full_from_lower(np.tril(d.double().cpu().numpy()))
            v = rng.standard_normal(A.shape[0])
            assert np.linalg.norm(A @ (X @ v) - v) / np.linalg.norm(v) <= ptol
        _check(hs[::97], ds[::97], tol)
