"""Host planner: the paper's task DAG (Table 1, Sec. 3) and the execution
plan of the persistent kernel (a topological order of the chain tasks)."""
import math
import os
import re

import pytest

from paper_1002_4057_gb300 import _lib as L

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_critical_path.txt")


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1002_4057_gb300 import build
    build.build()
    return L.lib()


def _eval(expr, t):
    e = re.sub(r"(\d)t", r"\1*t", expr.replace("^", "**"))
    v = eval(e, {"t": t})
    assert v == int(v)
    return int(v)


def _golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            parts = line.split()
            rows[parts[0]] = parts[1:]
    return rows


TS = list(range(2, 17)) + [24, 32, 48]


@pytest.mark.parametrize("t", TS)
def test_table1(t):
    g = _golden()
    _, inplace = L.spdinv_dag_critical_path(t, 0)
    _, oop = L.spdinv_dag_critical_path(t, L.SPDINV_DAG_OUT_OF_PLACE)
    for s in range(3):
        ip_expr, oop_expr = g["step%d" % (s + 1)]
        assert inplace[s] == _eval(ip_expr, t)
        assert oop[s] == _eval(oop_expr, t)


@pytest.mark.parametrize("t", TS)
def test_loop_reversal_uuu(t):
    g = _golden()
    _, ip = L.spdinv_dag_critical_path(t, L.SPDINV_DAG_UUU)
    _, oop = L.spdinv_dag_critical_path(t, L.SPDINV_DAG_UUU | L.SPDINV_DAG_OUT_OF_PLACE)
    assert ip[1] == _eval(g["uuu_step2"][0], t)
    assert oop[1] == _eval(g["uuu_step2"][1], t)
    # UUU never beats UDU
    _, udu = L.spdinv_dag_critical_path(t, 0)
    assert ip[1] >= udu[1]


@pytest.mark.parametrize("t", TS)
def test_pipelining(t):
    g = _golden()
    flags = L.SPDINV_DAG_OUT_OF_PLACE | L.SPDINV_DAG_RENAME_DIAG
    _, unp = L.spdinv_dag_critical_path(t, flags)
    _, pip = L.spdinv_dag_critical_path(t, flags | L.SPDINV_DAG_PIPELINE)
    assert unp[3] == _eval(g["oop_unpipelined"][0], t)
    assert pip[3] == _eval(g["oop_pipelined"][0], t)
    _, ipu = L.spdinv_dag_critical_path(t, 0)
    assert ipu[3] == _eval(g["inplace_unpipelined"][0], t)
    # pipelining never lengthens the path
    _, ipp = L.spdinv_dag_critical_path(t, L.SPDINV_DAG_PIPELINE)
    assert ipp[3] <= ipu[3]


def _alg1_counts(t):
    """Counts the tasks of each kind by walking Algorithm 1's loop nest."""
    c = [0] * 12
    for j in range(t):
        c[2] += j                      # SYRK(j,k), k<j
        c[0] += 1                      # POTRF(j)
        c[3] += (t - j - 1) * j        # GEMM(i,j,k)
        c[1] += t - j - 1              # TRSM(i,j)
    for j in range(t - 1, -1, -1):
        c[4] += 1                      # TRTRI(j)
        for i in range(t - 1, j, -1):
            c[5] += 1                  # TRMM(i,j) left
            c[6] += i - j - 1          # GEMM(i,j,k)
            c[7] += 1                  # TRMM(i,j) right
    for i in range(t):
        c[8] += i                      # TRMM(i,j), j<i
        c[9] += 1                      # LAUUM(i)
        c[10] += i * (t - i - 1)       # GEMM(i,j,k)
        c[11] += t - i - 1             # SYRK(i,k)
    return c



@pytest.mark.parametrize("t", [1, 2, 3, 4, 5, 8, 16, 33, 64])
def test_tree_reduced_chains(t):
    """The associative reduction of the commutative update chains (Sec. 3):
    m products into temporaries, a pairwise sum, one update of the tile.
    Step 3's chains read tiles that are all final when it starts, so alone it
    takes ceil(log2(t-1)) + 2 tasks (TRMM or LAUUM, the product level and the
    tree under the longest chain of t-1 products, the update) instead of t.
    Steps 1 and 2 receive their inputs one column at a time: a sequential
    chain ends one task after its last input, a tree ceil(log2 m) + 1 later,
    so trees there lengthen the path, and no tree variant beats the
    pipelined renamed chains (5t - 2)."""
    ren = L.SPDINV_DAG_OUT_OF_PLACE | L.SPDINV_DAG_RENAME_DIAG
    pip = ren | L.SPDINV_DAG_PIPELINE
    st, chains = L.spdinv_dag_critical_path(t, pip)
    assert st == 0 and chains[3] == max(5 * t - 2, 3)
    _, all_trees = L.spdinv_dag_critical_path(t, pip | L.SPDINV_DAG_TREE)
    _, s3_trees = L.spdinv_dag_critical_path(t, pip | L.SPDINV_DAG_TREE_STEP3)
    _, barrier_chains = L.spdinv_dag_critical_path(t, ren)
    _, barrier_s3 = L.spdinv_dag_critical_path(t, ren | L.SPDINV_DAG_TREE_STEP3)
    if t <= 2:  # no chain has two products
        assert all_trees == chains and s3_trees == chains
        return
    assert s3_trees[2] == math.ceil(math.log2(t - 1)) + 2
    assert s3_trees[:2] == chains[:2]
    assert all_trees[3] > chains[3] and s3_trees[3] >= chains[3]
    assert all_trees[0] >= chains[0] and all_trees[1] >= chains[1]
    if t >= 8:
        assert barrier_s3[3] < barrier_chains[3]



@pytest.mark.parametrize("t", [1, 2, 3, 4, 8, 16, 33, 64, 128])
def test_renaming_under_a_memory_budget(t):
    """C (the copy of L^{-1}) sharing B's storage (the copy of L) halves the
    renaming's extra memory; each step alone keeps its out-of-place path, but
    Step 3's copies into C now wait for Step 2's last reads of B, and the
    pipelined inversion takes 6t - 5 tasks (t >= 3) instead of 5t - 2 --
    barely under the barriered 6t - 3."""
    ren = L.SPDINV_DAG_OUT_OF_PLACE | L.SPDINV_DAG_RENAME_DIAG
    _, full = L.spdinv_dag_critical_path(t, ren | L.SPDINV_DAG_PIPELINE)
    _, shared = L.spdinv_dag_critical_path(t, ren | L.SPDINV_DAG_PIPELINE | L.SPDINV_DAG_SHARE_BC)
    _, barrier = L.spdinv_dag_critical_path(t, ren | L.SPDINV_DAG_SHARE_BC)
    assert shared[:3] == full[:3]
    if t >= 3:
        assert shared[3] == 6 * t - 5
        assert barrier[3] == 6 * t - 3
    assert full[3] <= shared[3] <= barrier[3]

def test_tree_flags_bound_t():
    assert L.spdinv_dag_critical_path(129, L.SPDINV_DAG_TREE)[0] == L.SPDINV_ERR_N
    assert L.spdinv_dag_critical_path(128, L.SPDINV_DAG_TREE_STEP3)[0] == 0

@pytest.mark.parametrize("t", [1, 2, 3, 7, 20])
def test_task_counts(t):
    st, c = L.spdinv_dag_task_counts(t)
    assert st == 0
    assert c == _alg1_counts(t)
    # every step does n^3/3 flops: leading terms sum to t^3 tile products
    assert c[3] == t * (t - 1) * (t - 2) // 6


def _deps(kind, i, j, t, steps):
    """Tasks whose output (kind, i, j) reads, written out from the chain
    definitions of the three steps (independent of the C++ planner)."""
    s1 = steps in (0, 1, 4)
    s2 = steps in (0, 2, 4)
    d = []
    D = (lambda q: [(0, q, q)]) if s1 else ((lambda q: [(2, q, q)]) if steps == 2 else (lambda q: []))
    Lt = (lambda a, b: [(1, a, b)]) if s1 else (lambda a, b: [])
    Xt = (lambda a, b: [(3, a, b)]) if s2 else (lambda a, b: [])
    if kind == 0:
        for k in range(j):
            d += Lt(j, k)
    elif kind == 1:
        for k in range(j):
            d += Lt(i, k) + Lt(j, k)
        d += D(j)
    elif kind == 3:
        d += D(i) + Lt(i, j) + D(j)
        for k in range(j + 1, i):
            d += Xt(i, k) + Lt(k, j)
    elif kind == 4:
        d += D(i)
        for k in range(i + 1, t):
            d += Xt(k, i)
    elif kind == 5:
        d += D(i) + Xt(i, j)
        for k in range(i + 1, t):
            d += Xt(k, i) + Xt(k, j)
    return d


@pytest.fixture(params=[L.SPDINV_PLAN_BOTTOM_LEVEL, L.SPDINV_PLAN_ALAP], ids=["bottom_level", "alap"])
def plan_order(request):
    old = L.spdinv_set_plan_order(request.param)
    yield request.param
    L.spdinv_set_plan_order(old)


@pytest.mark.parametrize("n,b,steps", [(512, 64, 0), (1000, 32, 0), (700, 64, 1), (700, 64, 2),
                                       (700, 64, 3), (700, 64, 4), (33, 32, 0), (1, 32, 0)])
def test_exec_plan_is_topological_and_complete(n, b, steps, plan_order):
    st, tasks, crit = L.spdinv_plan_tasks(n, b, steps)
    assert st == 0
    t = (n + b - 1) // b
    dec = [((e >> 28), (e >> 14) & 0x3FFF, e & 0x3FFF) for e in tasks]
    pos = {d: m for m, d in enumerate(dec)}
    assert len(pos) == len(dec)  # no duplicates
    expect = set()
    if steps in (0, 1, 4):
        expect |= {(0, j, j) for j in range(t)} | {(1, i, j) for i in range(t) for j in range(i)}
    if steps == 2:
        expect |= {(2, j, j) for j in range(t)}
    if steps in (0, 2, 4):
        expect |= {(3, i, j) for i in range(t) for j in range(i)}
    if steps in (0, 3, 4):
        expect |= {(4, i, i) for i in range(t)}
    if steps in (0, 3):
        expect |= {(5, i, j) for i in range(t) for j in range(i)}
    assert set(dec) == expect
    for m, (k, i, j) in enumerate(dec):
        for dep in _deps(k, i, j, t, steps):
            assert pos[dep] < m, (dec[m], dep)
    assert crit > 0



@pytest.mark.parametrize("steps", [0, 1, 2, 3, 4])
def test_fast_bottom_levels_match_the_edge_walk(steps):
    """Every plan (the full inversion 0, the steps alone 1-3, the selected
    inverse 4) is ordered by bottom levels computed from running maxima over
    the task grids in O(t^2); walking every dependency edge (O(t^3)) must give
    the same order, critical path and work."""
    for t in list(range(1, 41)) + [63, 64, 65, 97, 128]:
        st, (tasks, diff, cw) = L.spdinv_plan_check(t, steps)
        assert st == 0 and tasks > 0
        assert diff == 0 and cw == 0, (t, steps)

def test_exec_plan_puts_the_critical_path_first():
    _, tasks, _ = L.spdinv_plan_tasks(64 * 16, 64, 0)
    assert tasks[0] >> 28 == 0 and (tasks[0] & 0x3FFF) == 0  # Step-1 diagonal tile 0


@pytest.mark.parametrize("steps", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("t", [1, 2, 7, 40])
def test_schedule_model_bounds(steps, t):
    """spdinv_plan_simulate: one CTA runs the tickets back to back, so the
    makespan is the total work; any number of CTAs needs at least work / P
    and at most the task-level critical path once every task has a CTA."""
    st, (m1, w1, crit) = L.spdinv_plan_simulate(t, steps, 1)
    assert st == 0 and m1 == pytest.approx(w1, rel=1e-12)  # the same sum, in another order
    for P in (2, 5, 64):
        st, (m, w, _) = L.spdinv_plan_simulate(t, steps, P)
        assert st == 0 and w == w1 and w / P <= m * (1 + 1e-12) and m <= w * (1 + 1e-12)
    st, (minf, _, _) = L.spdinv_plan_simulate(t, steps, 10 ** 7)
    assert minf <= crit * (1 + 1e-12)


@pytest.mark.parametrize("t", [16, 64, 256])
def test_element_pipelined_critical_path_is_below_5t(t):
    """With a CTA for every task and each chain element waiting only for its
    own inputs, the full inversion's makespan stays under 5t tile products:
    the chain tasks keep the pipelined fine-grained DAG's critical path
    (5t - 2 unit tasks, Sec. 3), far below the task-level path (order t^2)."""
    st, (m, _, crit) = L.spdinv_plan_simulate(t, 0, 10 ** 7)
    assert st == 0
    assert 4 * t < m < 5 * t
    assert crit > t * t


def test_schedule_model_argument_errors():
    assert L.spdinv_plan_simulate(0, 0, 4)[0] == L.SPDINV_ERR_N
    assert L.spdinv_plan_simulate(4, 5, 4)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert L.spdinv_plan_simulate(4, 0, 0)[0] == L.SPDINV_ERR_UNSUPPORTED


@pytest.mark.parametrize("t,P,gain", [(64, 456, 0.08), (128, 912, 0.05), (128, 456, 0.02)])
def test_alap_order_keeps_more_ctas_busy(t, P, gain):
    """The ALAP ticket order (latest finish first, kept topological) against
    the bottom-level order in the schedule model: never worse, and clearly
    better where dependency waits cost most (n = 4096 at tiles 64 and 32)."""
    eff = {}
    for order in (L.SPDINV_PLAN_BOTTOM_LEVEL, L.SPDINV_PLAN_ALAP):
        old = L.spdinv_set_plan_order(order)
        try:
            st, (m, w, _) = L.spdinv_plan_simulate(t, 0, P)
        finally:
            L.spdinv_set_plan_order(old)
        assert st == 0
        eff[order] = w / (P * m)
    assert eff[L.SPDINV_PLAN_ALAP] >= eff[L.SPDINV_PLAN_BOTTOM_LEVEL] + gain, eff


@pytest.mark.parametrize("steps", [0, 1, 2, 3, 4])
def test_alap_order_runs_the_protocol_without_hazards(steps):
    old = L.spdinv_set_plan_order(L.SPDINV_PLAN_ALAP)
    try:
        for workers in (1, 7, 64):
            st, (done, total, errors, hazards, _) = L.spdinv_plan_emulate(17, workers, 3, max_delay_us=10,
                                                                          steps=steps)
            assert st == L.SPDINV_OK and done == total and errors == 0 and hazards == 0
    finally:
        L.spdinv_set_plan_order(old)


def test_plan_order_setter():
    old = L.spdinv_set_plan_order(L.SPDINV_PLAN_ALAP)
    try:
        assert L.spdinv_set_plan_order(7) == L.SPDINV_ERR_UNSUPPORTED
        assert L.spdinv_set_plan_order(L.SPDINV_PLAN_BOTTOM_LEVEL) == L.SPDINV_PLAN_ALAP
    finally:
        L.spdinv_set_plan_order(old)



@pytest.mark.parametrize("env,expected", [(None, 1), ("bottom_level", 0), ("0", 0), ("alap", 1)])
def test_plan_order_default_and_environment(env, expected):
    """The ALAP order is the default; SPDINV_PLAN_ORDER=bottom_level (or 0)
    selects the bottom-level order for the whole process."""
    import os
    import subprocess
    import sys
    e = dict(os.environ)
    e.pop("SPDINV_PLAN_ORDER", None)
    if env is not None:
        e["SPDINV_PLAN_ORDER"] = env
    code = ("from paper_1002_4057_gb300 import _lib as L; "
            "print(L.spdinv_set_plan_order(L.SPDINV_PLAN_BOTTOM_LEVEL))")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=e, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.strip().splitlines()[-1]) == expected
