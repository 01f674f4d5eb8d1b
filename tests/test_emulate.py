"""Host emulation of the persistent kernel's scheduling protocol
(spdinv_plan_emulate): worker threads take the plan's tickets, wait -- bounded
-- for their input tiles' flags in the kernel's order, store their output
tiles and publish them.  Every tile location records the task that last
stored it, and every read checks it (a read before the producer stored, or
of a tile of A after Step 3 overwrote it, is a hazard).  No GPU: this is the
race, deadlock, data-hazard and fault-injection coverage of the protocol on
the CPU, for every plan the kernel runs."""
import pytest

from paper_1002_4057_gb300 import _lib as L

ALL, POTRF, TRTRI, LAUUM, DIAG = range(5)


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1002_4057_gb300 import build
    build.build()
    return L.lib()


def _tasks(t, steps=ALL):
    tri, off = t * (t + 1) // 2, t * (t - 1) // 2
    return {ALL: tri + off + tri, POTRF: tri, TRTRI: tri, LAUUM: tri, DIAG: tri + off + t}[steps]


@pytest.mark.parametrize("t", [1, 2, 3, 8, 17, 40])
@pytest.mark.parametrize("workers", [1, 2, 5, 32, 256])
def test_every_worker_count_completes_without_hazards(t, workers):
    for seed in range(3):
        st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(t, workers, seed, max_delay_us=10)
        assert st == L.SPDINV_OK, (t, workers, seed)
        assert done == total == _tasks(t) and errors == 0 and hazards == 0


@pytest.mark.parametrize("steps", [POTRF, TRTRI, LAUUM, DIAG])
@pytest.mark.parametrize("t", [1, 2, 7, 24])
def test_every_plan_completes_without_hazards(steps, t):
    """The standalone steps (their other inputs staged before the launch)
    and the selected inverse."""
    for workers in (1, 3, 48):
        for seed in range(2):
            st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(t, workers, seed, max_delay_us=10,
                                                                          steps=steps)
            assert st == L.SPDINV_OK, (steps, t, workers, seed)
            assert done == total == _tasks(t, steps) and errors == 0 and hazards == 0


@pytest.mark.parametrize("steps", [ALL, POTRF, TRTRI, LAUUM, DIAG])
@pytest.mark.parametrize("t", [1, 5, 33])
def test_one_worker_never_waits(steps, t):
    """Tickets follow a topological order: a task's inputs are all published
    by tasks taken before it, so a lone worker finds every flag set."""
    st, (done, total, errors, hazards, longest_wait) = L.spdinv_plan_emulate(t, 1, 0, max_delay_us=0, steps=steps)
    assert st == L.SPDINV_OK and done == total and errors == hazards == 0 and longest_wait == 0


@pytest.mark.parametrize("steps,ticket", [(ALL, 1), (POTRF, 1), (DIAG, 1), (TRTRI, 2)])
def test_a_missing_wait_is_a_hazard(steps, ticket):
    """A task that reads without waiting (the skip_wait_task hook): the
    task with ticket 1 (2 in trtri, whose first two tickets invert diagonal
    tiles) reads a tile that an earlier ticket is still computing, and the
    check sees the read that came before the store."""
    seen = 0
    for seed in range(4):
        st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(8, 16, seed, max_delay_us=20000,
                                                                      steps=steps, skip_wait_task=ticket)
        assert st == L.SPDINV_OK and done == total and errors == 0
        seen += hazards > 0
    assert seen >= 3


def test_lauum_reads_only_staged_tiles():
    """spdinv_lauum stages X and its diagonal tiles before the launch, so its
    tasks wait for nothing and never race."""
    for skip in (0, 5, 20):
        st, (done, total, errors, hazards, longest_wait) = L.spdinv_plan_emulate(8, 16, 1, max_delay_us=2000,
                                                                                 steps=LAUUM, skip_wait_task=skip)
        assert st == L.SPDINV_OK and done == total and errors == hazards == 0 and longest_wait == 0


def test_a_lone_worker_hides_a_missing_wait():
    """The topological ticket order alone keeps one worker correct: the
    hazard needs concurrency, which is why the tests above run many."""
    for ticket in (1, 10, 50):
        st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(8, 1, 0, max_delay_us=0, skip_wait_task=ticket)
        assert st == L.SPDINV_OK and done == total and hazards == 0


def test_dropped_producer_ends_every_worker_with_a_timeout():
    """The fault_drop_task hook: the first task (the Cholesky of the first
    diagonal tile) never publishes; every task depends on it, so its consumers
    hit the wait limit, all workers stop, and the call returns."""
    st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(8, 16, 1, drop_task=0, wait_limit_s=0.2)
    assert st == L.SPDINV_ERR_TIMEOUT
    assert done < total and errors == 0 and hazards == 0


def test_dropped_task_without_consumers_is_harmless():
    """The last ticket belongs to Step 3, whose tasks publish nothing."""
    t = 6
    st, (done, total, _, hazards, _) = L.spdinv_plan_emulate(t, 8, 2, drop_task=_tasks(t) - 1, wait_limit_s=0.5)
    assert st == L.SPDINV_OK and done == total and hazards == 0


@pytest.mark.parametrize("drop", [3, 20, 50])
def test_dropped_task_midway_times_out_or_is_unread(drop):
    """A task in the middle of the plan: if anything reads its tile the run
    must end in a timeout, never hang; with an unread tile it completes."""
    t = 8
    st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(t, 12, 4, drop_task=drop, wait_limit_s=0.2)
    assert errors == 0 and hazards == 0
    assert (st == L.SPDINV_ERR_TIMEOUT and done < total) or (st == L.SPDINV_OK and done == total)
    _, tasks, _ = L.spdinv_plan_tasks(t * 32, 32, 0)
    kind = tasks[drop] >> 28
    if kind in (0, 1, 3):  # Steps 1 and 2 publish tiles that later tasks read
        assert st == L.SPDINV_ERR_TIMEOUT


def test_argument_errors():
    assert L.spdinv_plan_emulate(0, 4, 0)[0] == L.SPDINV_ERR_N
    assert L.spdinv_plan_emulate(4, 0, 0)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_emulate(4, 4, 0, wait_limit_s=0.0)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_emulate(4, 4, 0, steps=5)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_emulate(4, 4, 0, steps=-1)[0] == L.SPDINV_ERR_UNSUPPORTED


# ---- execution variants (the study of Sec. 3 on the GPU) -------------------
UUU, SHARE, INPLACE, SPLIT = (L.SPDINV_VARIANT_UUU, L.SPDINV_VARIANT_SHARE_BC, L.SPDINV_VARIANT_INPLACE,
                              L.SPDINV_VARIANT_SPLIT3)
VARIANTS = [(UUU, 0), (SHARE, 0), (INPLACE, 0), (UUU | SHARE, 0), (UUU | INPLACE, 0), (SPLIT, 1), (SPLIT, 2),
            (SPLIT, 5), (SPLIT | UUU, 3)]


def _variant_tasks(t, var, seg):
    n = _tasks(t)
    if var & SPLIT:  # one task per extra segment of each Step-3 chain longer than seg
        for i in range(t):
            m = t - 1 - i
            if m > seg:
                n += (i + 1) * (-(-m // seg) - 1)
    return n


@pytest.mark.parametrize("var,seg", VARIANTS)
@pytest.mark.parametrize("t", [1, 2, 3, 6, 11, 24])
@pytest.mark.parametrize("workers", [1, 3, 16, 96])
def test_variant_plans_complete_without_hazards(var, seg, t, workers):
    """With C in B's slots or a single store, a version of a tile is stored
    only after every read of the previous one: the emulator records each
    tile's writer and counts each read, so a read of an overwritten tile is a
    hazard and a read count that differs from the one the writers wait for is
    a protocol error.  One worker never waits, which shows the ticket order
    is topological over the write-after-read edges too."""
    for seed in range(2):
        st, (done, total, errors, hazards, longest) = L.spdinv_plan_emulate_variant(
            t, var, workers, seed, split_segment=seg, max_delay_us=8)
        assert st == L.SPDINV_OK, (var, seg, t, workers, seed)
        assert done == total == _variant_tasks(t, var, seg)
        assert errors == 0 and hazards == 0
        if workers == 1:
            assert longest == 0


@pytest.mark.parametrize("var", [SHARE, INPLACE])
def test_variant_dropped_producer_times_out(var):
    """A task that never publishes (the kernel's fault hook) ends every worker
    with a timeout, also where writers wait on read counts."""
    st, (done, total, _, _, _) = L.spdinv_plan_emulate_variant(8, var, 8, 1, drop_task=3, wait_limit_s=0.3,
                                                                max_delay_us=2)
    assert st == L.SPDINV_ERR_TIMEOUT and done < total


def test_variant_rejects_unsupported_combinations():
    out = L.spdinv_plan_emulate_variant(5, SPLIT | SHARE, 2, 0, split_segment=2)
    assert out[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_emulate_variant(5, SPLIT | INPLACE, 2, 0, split_segment=2)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_emulate_variant(5, 64, 2, 0)[0] == L.SPDINV_ERR_UNSUPPORTED
