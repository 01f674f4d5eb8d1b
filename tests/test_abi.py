"""The C-ABI library loads, exports every symbol include/spdinv.h declares,
and rejects bad arguments synchronously (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1002_4057_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1002_4057_gb300 import build
    build.build()
    return L.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "spdinv.h")).read()
    return sorted(set(re.findall(r"SPDINV_API\s+[\w\s\*]+?\b(spdinv_\w+)\s*\(", text)))


def test_header_declares_the_three_steps_and_the_pipelined_whole():
    names = declared_symbols()
    for n in ("spdinv_potrf", "spdinv_trtri", "spdinv_lauum", "spdinv_potri", "spdinv_potri_batched"):
        assert n in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, n


def test_version(lib):
    assert L.spdinv_version() >= 10000


@pytest.mark.parametrize("fn", ["spdinv_potrf", "spdinv_trtri", "spdinv_potri"])
def test_argument_errors(lib, fn):
    f = getattr(L, fn)
    assert f(-1, 0, 1, None, None) == L.SPDINV_ERR_N
    assert f(10, 8, 5, None, None) == L.SPDINV_ERR_LDA
    assert f(10, None, 10, None, None) == L.SPDINV_ERR_NULL
    assert f(0, None, 1, None, None) == L.SPDINV_OK  # quick return, nothing queued


def test_lauum_argument_errors(lib):
    assert L.spdinv_lauum(-3, 8, 1, None) == L.SPDINV_ERR_N
    assert L.spdinv_lauum(4, 8, 3, None) == L.SPDINV_ERR_LDA


def test_unsupported_tile(lib):
    o = L.spdinv_opts(48, 0, 0, 0, 0.0, -1)
    assert L.spdinv_potri_ex(100, 8, 100, o, None, None) == L.SPDINV_ERR_UNSUPPORTED


@pytest.mark.parametrize("order,residual", [(1, 0), (9, 0), (-2, 0), (3, 1), (3, 2)])
def test_unsupported_refine_order(lib, order, residual):
    """Correction orders outside 2..8, and orders above 2 on the residual
    paths that have only the Newton-Schulz step, are rejected before any
    device work (the pointer is never touched)."""
    o = L.spdinv_opts(64, 0, 1, 1, 0.0, -1, residual, order)
    assert L.spdinv_potri_ex(100, 8, 100, o, None, None) == L.SPDINV_ERR_UNSUPPORTED


def test_planner_queries_need_no_gpu(lib):
    st, cp = L.spdinv_dag_critical_path(4, 0)
    assert st == 0 and cp[:3] == [10, 9, 10]
    assert L.spdinv_dag_critical_path(0, 0)[0] == L.SPDINV_ERR_N


def _ints(*v):
    a = (ctypes.c_int * max(len(v), 1))(*v)
    return a, ctypes.addressof(a)


FAKE = 4096  # a non-NULL pointer that no argument check may dereference


def test_potri_ex_option_errors(lib):
    """Every option is checked before any device work."""
    mixed = L.SPDINV_PREC_MIXED_FP32
    bad = [
        L.spdinv_opts(48, 0, mixed, 1, 0.0, -1, 0, 0),   # tile
        L.spdinv_opts(64, 0, mixed, 17, 0.0, -1, 0, 0),  # correction steps
        L.spdinv_opts(64, 0, mixed, -1, 0.0, -1, 0, 0),
        L.spdinv_opts(64, 0, mixed, 1, 0.0, -1, 5, 0),   # residual path
        L.spdinv_opts(64, 0, mixed, 1, 0.0, -1, -1, 0),
        L.spdinv_opts(64, 0, 4, 1, 0.0, -1, 0, 0),       # unknown precision
        L.spdinv_opts(64, 0, 7, 1, 0.0, -1, 0, 0),
        L.spdinv_opts(64, 0, mixed, 1, 0.0, -1, 0, 0, 0, 0, 2),   # diagonal precision
        L.spdinv_opts(64, 0, mixed, 1, 0.0, -1, 0, 0, 0, 0, -1),
    ]
    for o in bad:
        assert L.spdinv_potri_ex(100, FAKE, 100, o, None, None) == L.SPDINV_ERR_UNSUPPORTED
    o = L.spdinv_opts(64, 0, mixed, 1, 0.0, -1, 0, 0)
    assert L.spdinv_potri_ex(100, FAKE, 99, o, None, None) == L.SPDINV_ERR_LDA
    assert L.spdinv_potri_ex(100, None, 100, o, None, None) == L.SPDINV_ERR_NULL
    assert L.spdinv_potri_ex(-1, FAKE, 100, o, None, None) == L.SPDINV_ERR_N
    assert L.spdinv_potri_ex(0, None, 1, o, None, None) == L.SPDINV_OK


def test_tile_grid_limit(lib):
    """The plan encodes tile indices in 14 bits: t = ceil(n / b) <= 16383."""
    o = L.spdinv_opts(32, 0, 0, 0, 0.0, -1, 0, 0)
    n = 16384 * 32
    assert L.spdinv_potri_ex(n, FAKE, n, o, None, None) == L.SPDINV_ERR_N
    assert L.spdinv_potrf(2 * n, FAKE, 2 * n, None, None) == L.SPDINV_ERR_N  # default tile 64


def test_potri_diag_and_noalloc_errors(lib):
    assert L.spdinv_potri_diag(10, FAKE, 10, None, None, None) == L.SPDINV_ERR_NULL
    assert L.spdinv_potri_diag(10, FAKE, 9, FAKE, None, None) == L.SPDINV_ERR_LDA
    assert L.spdinv_potri_diag(-1, FAKE, 9, FAKE, None, None) == L.SPDINV_ERR_N
    assert L.spdinv_potri_diag(0, None, 1, None, None, None) == L.SPDINV_OK
    assert L.spdinv_potri_noalloc(1025, FAKE, 1025, None, None) == L.SPDINV_ERR_N
    assert L.spdinv_potri_noalloc(-1, FAKE, 1, None, None) == L.SPDINV_ERR_N
    assert L.spdinv_potri_noalloc(10, FAKE, 9, None, None) == L.SPDINV_ERR_LDA
    assert L.spdinv_potri_noalloc(10, None, 10, None, None) == L.SPDINV_ERR_NULL
    assert L.spdinv_potri_noalloc(0, None, 1, None, None) == L.SPDINV_OK


def test_inverse_residual_errors(lib):
    f = L.spdinv_inverse_residual
    assert f(-1, FAKE, 1, FAKE, FAKE, 0, None) == L.SPDINV_ERR_N
    assert f(8, FAKE, 7, FAKE, FAKE, 0, None) == L.SPDINV_ERR_LDA
    for args in ((None, FAKE, FAKE), (FAKE, None, FAKE), (FAKE, FAKE, None)):
        assert f(8, args[0], 8, args[1], args[2], 0, None) == L.SPDINV_ERR_NULL
    assert f(8, FAKE, 8, FAKE, FAKE, 3, None) == L.SPDINV_ERR_UNSUPPORTED
    assert f(0, None, 1, None, None, 0, None) == L.SPDINV_OK


@pytest.mark.parametrize("fn", ["spdinv_potri_batched", "spdinv_spotri_batched"])
def test_batched_errors(lib, fn):
    f = getattr(L, fn)
    n, pn = _ints(16, 32, 5)
    ld, pld = _ints(16, 32, 5)
    assert f(-1, pn, FAKE, pld, None, None) == L.SPDINV_ERR_N
    assert f(0, None, None, None, None, None) == L.SPDINV_OK
    assert f(3, None, FAKE, pld, None, None) == L.SPDINV_ERR_NULL
    assert f(3, pn, None, pld, None, None) == L.SPDINV_ERR_NULL
    assert f(3, pn, FAKE, None, None, None) == L.SPDINV_ERR_NULL
    big, pbig = _ints(16, 4097, 5)
    assert f(3, pbig, FAKE, pbig, None, None) == L.SPDINV_ERR_N
    neg, pneg = _ints(16, -1, 5)
    assert f(3, pneg, FAKE, pld, None, None) == L.SPDINV_ERR_N
    short, pshort = _ints(16, 31, 5)
    assert f(3, pn, FAKE, pshort, None, None) == L.SPDINV_ERR_LDA


@pytest.mark.parametrize("fn", ["spdinv_potri_backward", "spdinv_spotri_backward"])
def test_backward_errors(lib, fn):
    f = getattr(L, fn)
    n = 8

    def call(batch, n, X=FAKE, G=FAKE, R=FAKE, ldx=8, ldg=8, ldr=8):
        return f(batch, n, X, ldx, n * ldx, G, ldg, n * ldg, R, ldr, n * ldr, None)
    assert call(-1, n) == L.SPDINV_ERR_N
    assert call(1, -1) == L.SPDINV_ERR_N
    for k in ("ldx", "ldg", "ldr"):
        assert call(1, n, **{k: n - 1}) == L.SPDINV_ERR_LDA
    for k in ("X", "G", "R"):
        assert call(1, n, **{k: None}) == L.SPDINV_ERR_NULL
    assert call(65536, n) == L.SPDINV_ERR_N
    assert call(0, n, X=None, G=None, R=None) == L.SPDINV_OK
    assert call(3, 0, X=None, G=None, R=None) == L.SPDINV_OK


@pytest.mark.parametrize("fn", ["spdinv_mirror_lower", "spdinv_smirror_lower"])
def test_mirror_errors(lib, fn):
    f = getattr(L, fn)
    assert f(-1, 8, FAKE, 8, 64, None) == L.SPDINV_ERR_N
    assert f(1, -8, FAKE, 8, 64, None) == L.SPDINV_ERR_N
    assert f(65536, 8, FAKE, 8, 64, None) == L.SPDINV_ERR_N
    assert f(1, 8, FAKE, 7, 64, None) == L.SPDINV_ERR_LDA
    assert f(1, 8, None, 8, 64, None) == L.SPDINV_ERR_NULL
    assert f(0, 8, None, 8, 64, None) == L.SPDINV_OK
    assert f(2, 0, None, 1, 0, None) == L.SPDINV_OK


def test_batched_tiles_needs_an_output(lib):
    assert L._call("spdinv_batched_tiles", 0, None) == L.SPDINV_ERR_NULL


# ------------------------------------------------------- caller workspace
def _ws(n, routine, opts=None):
    st, nbytes = L.spdinv_workspace_size(n, routine, opts)
    assert st == L.SPDINV_OK, st
    return nbytes


def test_workspace_size_fp64_layout(lib):
    """n = 100, tile 32: t = 4; status words and flags 4 * (4 + 2*16 + 4)
    bytes rounded up to 256; B and C hold t(t-1)/2 = 6 tiles of 32*32*8 =
    8192 bytes; D holds 4 tiles."""
    tiles6, tiles4 = 6 * 8192, 4 * 8192
    assert _ws(100, L.SPDINV_ROUTINE_POTRI) == 256 + 2 * tiles6 + tiles4
    assert _ws(100, L.SPDINV_ROUTINE_POTRI_DIAG) == 256 + 2 * tiles6 + tiles4
    assert _ws(100, L.SPDINV_ROUTINE_TRTRI) == 256 + 2 * tiles6 + tiles4
    assert _ws(100, L.SPDINV_ROUTINE_POTRF) == 256 + tiles6 + tiles4  # no C
    assert _ws(100, L.SPDINV_ROUTINE_LAUUM) == 256 + tiles6 + tiles4  # no B
    o = L.spdinv_opts(64, 0, 0, 0, 0.0, -1, 0, 0)  # tile 64: t = 2, one 32 KB tile in B and C
    assert _ws(100, L.SPDINV_ROUTINE_POTRI, o) == 256 + 2 * 32768 + 2 * 32768
    # the benchmark's size: t = 512, flags 4 * 524804 bytes -> 2099456; 130816 tiles in B and C
    assert _ws(16384, L.SPDINV_ROUTINE_POTRI) == 2099456 + 2 * 130816 * 8192 + 512 * 8192
    assert _ws(0, L.SPDINV_ROUTINE_POTRI) == 0


def test_workspace_size_mixed_and_residual_layout(lib):
    """Mixed, n = 100, tile 64: t = 2; FP32 tiles of 64 x 65 floats = 16640
    bytes (one in B, one in C, two in D); X is 100*100*8 = 80000 bytes,
    rounded to 80128; with correction steps three such matrices and 23 BF16
    planes of 256 x 256 (7 + 7 slices for R, 5 of R, 4 of the terms) plus
    256 * (8 + 16) bytes of scales and 1024 bytes of pad."""
    mixed = L.SPDINV_PREC_MIXED_FP32
    base = 256 + 2 * 16640 + 33280
    o = L.spdinv_opts(64, 0, mixed, 0, 0.0, -1, 0, 0)
    assert _ws(100, L.SPDINV_ROUTINE_POTRI, o) == base + 80128
    o = L.spdinv_opts(64, 0, mixed, 1, 0.0, -1, 0, 3)
    planes = 23 * 65536 * 2 + 256 * 24 + 1024
    assert _ws(100, L.SPDINV_ROUTINE_POTRI, o) == base + 3 * 80128 + planes
    # the automatic tile is 32 up to n = 8192 and 64 above
    for n, b in ((100, 32), (8192, 32), (8193, 64)):
        assert _ws(n, L.SPDINV_ROUTINE_POTRI, L.spdinv_opts(0, 0, mixed, 0, 0.0, -1, 0, 0)) == \
            _ws(n, L.SPDINV_ROUTINE_POTRI, L.spdinv_opts(b, 0, mixed, 0, 0.0, -1, 0, 0))
    # the residual alone: 256 bytes of status words, plus 2 x 7 slice planes,
    # 256 ints and 256 64-bit maxima per side and 1024 bytes of pad when emulated
    r = L.SPDINV_ROUTINE_INVERSE_RESIDUAL
    assert _ws(100, r, L.spdinv_opts(0, 0, 0, 0, 0.0, -1, L.SPDINV_RESIDUAL_FP64, 0)) == 256
    assert _ws(100, r) == 256 + 14 * 65536 * 2 + 2 * 256 * 4 + 2 * 256 * 8 + 1024


def test_workspace_size_errors(lib):
    f = L.spdinv_workspace_size
    assert f(-1, 0)[0] == L.SPDINV_ERR_N
    assert f(10, 6)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert f(10, -1)[0] == L.SPDINV_ERR_UNSUPPORTED
    assert f(10, 0, L.spdinv_opts(48, 0, 0, 0, 0.0, -1, 0, 0))[0] == L.SPDINV_ERR_UNSUPPORTED
    assert f(10, 0, L.spdinv_opts(0, 0, 4, 0, 0.0, -1, 0, 0))[0] == L.SPDINV_ERR_UNSUPPORTED  # unknown precision
    assert f(10, 0, L.spdinv_opts(0, 0, 2, 0, 0.0, -1, 0, 0))[0] == L.SPDINV_OK  # BF16x3
    assert f(10, 0, L.spdinv_opts(0, 0, 3, 0, 0.0, -1, 0, 0))[0] == L.SPDINV_OK  # 3xTF32
    assert f(10, 0, L.spdinv_opts(0, 0, 1, 1, 0.0, -1, 0, 9))[0] == L.SPDINV_ERR_UNSUPPORTED  # order 9
    assert f(10, 5, L.spdinv_opts(0, 0, 0, 0, 0.0, -1, 7, 0))[0] == L.SPDINV_ERR_UNSUPPORTED  # residual path
    assert f(32 * 16384, 0, L.spdinv_opts(32, 0, 0, 0, 0.0, -1, 0, 0))[0] == L.SPDINV_ERR_N
    assert L._call("spdinv_workspace_size", 10, 0, None, None) == L.SPDINV_ERR_NULL


def test_set_workspace_rejects_a_misaligned_buffer(lib):
    assert L.spdinv_set_workspace(4096 + 16, 1 << 20) == L.SPDINV_ERR_WORKSPACE


def _run_py(code, **env):
    import subprocess
    import sys
    e = dict(os.environ)
    e.update(env)
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=e, capture_output=True, text=True,
                          timeout=120, check=True)


_CALLS = ("from paper_1002_4057_gb300 import _lib as L\n"
          "L.spdinv_potri(-1, None, 1, None, None)\n"
          "L.spdinv_potri(0, None, 1, None, None)\n"
          "L.spdinv_potri_batched(-2, None, None, None, None, None)\n")


def test_log_flag(lib):
    """SPDINV_LOG=1: one stderr line per call that returns an error status;
    SPDINV_LOG=2: every call; unset: nothing."""
    quiet = _run_py(_CALLS)
    assert "[spdinv]" not in quiet.stderr
    errs = [l for l in _run_py(_CALLS, SPDINV_LOG="1").stderr.splitlines() if l.startswith("[spdinv]")]
    assert errs == ["[spdinv] spdinv_potri n=-1: SPDINV_ERR_N",
                    "[spdinv] spdinv_potri_batched batch=-2: SPDINV_ERR_N"]
    every = [l for l in _run_py(_CALLS, SPDINV_LOG="2").stderr.splitlines() if l.startswith("[spdinv]")]
    assert every[1] == "[spdinv] spdinv_potri n=0: SPDINV_OK" and len(every) == 3


def test_tile_override(lib):
    """SPDINV_TILE=64 replaces the default tile 32 at n = 16384 (t = 256:
    flags 4 * 131332 bytes -> 525568; 32640 tiles of 32 KB in B and C)."""
    code = ("from paper_1002_4057_gb300 import _lib as L\n"
            "print(L.spdinv_workspace_size(16384, 0)[1])\n")
    assert int(_run_py(code, SPDINV_TILE="64").stdout) == 525568 + 2 * 32640 * 32768 + 256 * 32768
    assert int(_run_py(code, SPDINV_TILE="48").stdout) == _ws(16384, L.SPDINV_ROUTINE_POTRI)  # ignored


def test_debug_flags_round_trip(lib):
    old = L.spdinv_set_debug_flags(L.SPDINV_DEBUG_POISON)
    try:
        assert L.spdinv_set_debug_flags(0) == L.SPDINV_DEBUG_POISON
        assert L.spdinv_set_debug_flags(0) == 0
    finally:
        L.spdinv_set_debug_flags(old)


def test_status_names_match_the_binding(lib):
    for code, name in L.STATUS_NAMES.items():
        assert L.spdinv_status_name(code) == name
    assert L.spdinv_status_name(-99) == "unknown status"


@pytest.mark.parametrize("wide", [1, 0])
@pytest.mark.parametrize("lower", [0, 1])
def test_slice_gemm_tile_order_is_a_bijection(lib, lower, wide):
    """The slice GEMM launches one CTA per output tile in a grouped raster
    (groups of 8 row blocks for the full 128 x 256 grid, 16 for its lower
    tiles and for the 128 x 128 grid).  Replayed on the host through the
    kernels' own index functions, every launch index takes a distinct tile of
    the grid (only tiles holding an entry on or below the diagonal when
    lower), and every such tile is taken -- including grids that end in a
    partial group."""
    for n in (1, 255, 256, 257, 1030, 2300, 4096, 5000, 16384, 20000, 32768):
        npad = (n + 255) // 256 * 256
        tb_m = npad // 128
        cols = 256 if wide else 128
        tb_n = npad // cols
        st, bm, bn = L.spdinv_slice_tile_order(n, lower, wide)
        assert st == 0
        want = {(r, c) for r in range(tb_m) for c in range(tb_n)
                if not lower or c * cols <= r * 128 + 127}
        assert len(bm) == len(want), (n, len(bm), len(want))
        assert set(zip(bm, bn)) == want, n


def test_slice_gemm_tile_order_groups(lib):
    """The full 128 x 256 grid at n = 16384 (128 x 64 tiles) runs groups of 8
    row blocks column by column: the first 8 launch indices are column 0 of
    rows 0-7, and each group covers its 8 rows before the next starts."""
    st, bm, bn = L.spdinv_slice_tile_order(16384, 0, 1)
    assert st == 0
    assert list(zip(bm[:9], bn[:9])) == [(r, 0) for r in range(8)] + [(0, 1)]
    per_group = 8 * 64
    for g in range(128 // 8):
        assert set(bm[g * per_group:(g + 1) * per_group]) == set(range(8 * g, 8 * g + 8))


def test_slice_gemm_tile_order_errors(lib):
    cnt = ctypes.c_int(0)
    assert L._call("spdinv_slice_tile_order", 0, 0, 1, None, None, ctypes.addressof(cnt)) == L.SPDINV_ERR_N
    assert L._call("spdinv_slice_tile_order", (1 << 20) + 1, 0, 1, None, None, ctypes.addressof(cnt)) == L.SPDINV_ERR_N
    assert L._call("spdinv_slice_tile_order", 100, 0, 1, None, None, None) == L.SPDINV_ERR_NULL
    a = (ctypes.c_int * 4)()
    assert L._call("spdinv_slice_tile_order", 100, 0, 1, ctypes.addressof(a), None,
                   ctypes.addressof(cnt)) == L.SPDINV_ERR_NULL
