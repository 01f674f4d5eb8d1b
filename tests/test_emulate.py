"""Host emulation of the persistent kernel's scheduling protocol
(spdinv_plan_emulate): worker threads take the plan's tickets, wait -- bounded
-- for their input tiles' flags in the kernel's order and publish their
outputs.  No GPU: this is the race, deadlock and fault-injection coverage of
the protocol on the CPU."""
import pytest

from paper_1002_4057_gb300 import _lib as L


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1002_4057_gb300 import build
    build.build()
    return L.lib()


def _tasks(t):
    # full inversion: t(t+1)/2 tasks in Steps 1 and 3, t(t-1)/2 in Step 2
    return t * (t + 1) + t * (t - 1) // 2


@pytest.mark.parametrize("t", [1, 2, 3, 8, 17, 40])
@pytest.mark.parametrize("workers", [1, 2, 5, 32, 256])
def test_every_worker_count_completes(t, workers):
    for seed in range(3):
        st, (done, total, errors, _) = L.spdinv_plan_emulate(t, workers, seed, max_delay_us=10)
        assert st == L.SPDINV_OK, (t, workers, seed)
        assert done == total == _tasks(t) and errors == 0


@pytest.mark.parametrize("t", [1, 5, 33])
def test_one_worker_never_waits(t):
    """Tickets follow a topological order: a task's inputs are all published
    by tasks taken before it, so a lone worker finds every flag set."""
    st, (done, total, errors, longest_wait) = L.spdinv_plan_emulate(t, 1, 0, max_delay_us=0)
    assert st == L.SPDINV_OK and done == total and longest_wait == 0


def test_dropped_producer_ends_every_worker_with_a_timeout():
    """The fault_drop_task hook: the first task (the Cholesky of the first
    diagonal tile) never publishes; every task depends on it, so its consumers
    hit the wait limit, all workers stop, and the call returns."""
    st, (done, total, errors, _) = L.spdinv_plan_emulate(8, 16, 1, drop_task=0, wait_limit_s=0.2)
    assert st == L.SPDINV_ERR_TIMEOUT
    assert done < total and errors == 0


def test_dropped_task_without_consumers_is_harmless():
    """The last ticket belongs to Step 3, whose tasks publish nothing."""
    t = 6
    st, (done, total, errors, _) = L.spdinv_plan_emulate(t, 8, 2, drop_task=_tasks(t) - 1, wait_limit_s=0.5)
    assert st == L.SPDINV_OK and done == total


@pytest.mark.parametrize("drop", [3, 20, 50])
def test_dropped_task_midway_times_out_or_is_unread(drop):
    """A task in the middle of the plan: if anything reads its tile the run
    must end in a timeout, never hang; with an unread tile it completes."""
    t = 8
    st, (done, total, errors, _) = L.spdinv_plan_emulate(t, 12, 4, drop_task=drop, wait_limit_s=0.2)
    assert errors == 0
    assert (st == L.SPDINV_ERR_TIMEOUT and done < total) or (st == L.SPDINV_OK and done == total)
    _, tasks, _ = L.spdinv_plan_tasks(t * 32, 32, 0)
    kind = tasks[drop] >> 28
    if kind in (0, 1, 3):  # Steps 1 and 2 publish tiles that later tasks read
        assert st == L.SPDINV_ERR_TIMEOUT


def test_argument_errors():
    assert L.spdinv_plan_emulate(0, 4, 0)[0] == L.SPDINV_ERR_N
    assert L.spdinv_plan_emulate(4, 0, 0)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_emulate(4, 4, 0, wait_limit_s=0.0)[0] == L.SPDINV_ERR_UNSUPPORTED
