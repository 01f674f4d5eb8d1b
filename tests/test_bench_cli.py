"""bench.py on the CPU: it parses, prints its help, and its reference arm
(the oracle on the host cores) prints one JSON line with the contract's keys.
The GPU arms run on a GB300 only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_help():
    r = _bench("--help")
    assert r.returncode == 0 and "--workload" in r.stdout and "--plan-order" in r.stdout


def test_reference_arm_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    for key in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["value"] > 0


def test_graft_entry_exposes_build_and_smoke():
    sys.path.insert(0, ROOT)
    try:
        import __graft_entry__ as g
    finally:
        sys.path.remove(ROOT)
    assert callable(g.build) and callable(g.smoke)
