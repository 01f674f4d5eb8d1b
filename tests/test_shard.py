"""Multi-GPU split of a batch (spdinv_batch_shard): host-only, so it is tested
on the CPU -- its properties, against brute force on tiny batches, and as two
gloo ranks that each take their share and check, by exchanging them, that the
shares are disjoint, complete and agree."""
import itertools
import socket

import numpy as np
import pytest

import spd_inputs as si
from paper_1002_4057_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    from paper_1002_4057_gb300 import build
    build.build()
    return L.lib()


def _work(sizes):
    return np.asarray(sizes, dtype=np.float64) ** 3


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_split_is_a_partition_and_balanced(lib, world):
    sizes = si.batch_sizes(4096, 16, 256, seed=si.SEED_BASE + 3)
    st, owner, load = L.spdinv_batch_shard(sizes, world)
    assert st == 0
    owner = np.asarray(owner)
    assert owner.min() >= 0 and owner.max() < world
    w = _work(sizes)
    per = np.array([w[owner == r].sum() for r in range(world)])
    assert np.allclose(per, load)
    assert np.isclose(per.sum(), w.sum())
    # longest-processing-time bound: makespan <= 4/3 of a lower bound on the optimum
    opt_lb = max(w.sum() / world, w.max())
    assert per.max() <= 4.0 / 3.0 * opt_lb
    # on this many small jobs the split is nearly even
    assert per.max() <= 1.01 * w.sum() / world


def test_split_is_deterministic_and_follows_lpt_order(lib):
    sizes = [5, 9, 9, 3, 7, 1, 9]
    st, owner, load = L.spdinv_batch_shard(sizes, 2)
    assert st == 0
    # by hand: 9(i1)->0, 9(i2)->1, 9(i6)->0 (tie, lower rank), then 7, 5, 3, 1
    # all to rank 1, which stays the lighter one
    assert owner == [1, 0, 1, 1, 1, 1, 0]
    assert load == [729.0 * 2, 729.0 + 343 + 125 + 27 + 1]
    assert L.spdinv_batch_shard(sizes, 2)[1] == owner


@pytest.mark.parametrize("seed", range(6))
def test_split_within_four_thirds_of_brute_force(lib, seed):
    r = np.random.default_rng(seed)
    sizes = list(r.integers(1, 40, size=7))
    w = _work(sizes)
    for world in (2, 3):
        st, owner, _ = L.spdinv_batch_shard(sizes, world)
        assert st == 0
        got = max(w[np.asarray(owner) == q].sum() for q in range(world))
        best = min(max(w[np.asarray(a) == q].sum() for q in range(world))
                   for a in itertools.product(range(world), repeat=len(sizes)))
        assert got <= 4.0 / 3.0 * best + 1e-9


def test_split_argument_errors(lib):
    assert L.spdinv_batch_shard([4, 5], 0)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_batch_shard([4, -1], 2)[0] == L.SPDINV_ERR_N
    st, owner, load = L.spdinv_batch_shard([], 3)
    assert st == 0 and owner == [] and load == [0.0, 0.0, 0.0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, count, q):
    import torch.distributed as dist
    try:
        dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
        sizes = si.batch_sizes(count, 16, 256, seed=si.SEED_BASE + 3)
        st, owner, load = L.spdinv_batch_shard(sizes, world)
        mine = [k for k in range(count) if owner[k] == rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, {"owner": owner, "mine": mine, "work": float(_work(sizes[mine]).sum())})
        # the bench's aggregate: total work of all ranks over the slowest rank's time
        import torch
        t = torch.tensor([1.0 + rank])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        q.put((rank, st, gathered, float(t.item())))
        dist.destroy_process_group()
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e), None, None))


def test_two_gloo_ranks_take_disjoint_complete_shares():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, count, port = 2, 600, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, count, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, st, gathered, tmax in res:
        assert st == 0, st
        assert tmax == float(world)
        owners = [g["owner"] for g in gathered]
        assert all(o == owners[0] for o in owners)  # every rank computed the same split
        shares = [set(g["mine"]) for g in gathered]
        assert not (shares[0] & shares[1])
        assert shares[0] | shares[1] == set(range(count))
        works = [g["work"] for g in gathered]
        assert max(works) <= 1.02 * sum(works) / world
