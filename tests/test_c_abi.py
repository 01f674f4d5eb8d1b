"""include/spdinv.h is a C header: a plain C99 program (tests/c/abi_check.c)
compiles against it with gcc -std=c99 -Wall -Werror, links libspdinv.so and
calls the entry points that need no GPU.  No Python between the caller and
the library."""
import os
import shutil
import subprocess

import pytest

from paper_1002_4057_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


def test_plain_c_caller(tmp_path):
    if shutil.which("gcc") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("gcc or the CUDA headers are missing")
    lib = build.build()
    exe = tmp_path / "abi_check"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), "-isystem", CUDA_INC,
                           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-o", str(exe),
                           "-L", os.path.dirname(lib), "-lspdinv", "-Wl,-rpath," + os.path.dirname(lib)])
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout
    got = dict(line.split(" ", 1) for line in out.strip().splitlines())
    assert int(got["version"]) >= 10000
    assert got["potri_n"] == "-1" and got["potri_lda"] == "-2" and got["potri_null"] == "-3"
    assert got["potri_empty"] == "0" and got["potri_ex_tile"] == "-6"
    assert got["critical"] == "0 10 9 10"
    assert got["plan"] == "0 26"  # t = 4: 10 + 6 + 10 chain tasks (Steps 1, 2, 3)
    assert got["first_task"] == "0"  # the Cholesky of tile (0, 0) comes first
    assert got["plan_check"] == "0 0 0"
    # sizes 5, 9, 9, 3, 7 on two ranks, largest first: 9 -> 0, 9 -> 1, 7 -> 0
    # (tie, lower rank), 5 -> 1, 3 -> 1; loads 729 + 343 and 729 + 125 + 27
    assert got["shard"] == "0 1 0 1 1 0 1072 881"
    # n = 2300 pads to 2304: 18 row blocks of 128, the lower 128 x 256 tiles 9 * 10
    assert got["slice_tiles"] == "0 90"
    # the binding's spdinv_opts has the header's layout
    from paper_1002_4057_gb300 import _lib as L
    import ctypes
    assert int(got["opts_size"]) == ctypes.sizeof(L.spdinv_opts)
    offs = [getattr(L.spdinv_opts, f).offset for f, _ in L.spdinv_opts._fields_]
    assert [int(v) for v in got["opts_offsets"].split()] == offs
