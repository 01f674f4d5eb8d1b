"""The C-ABI library loads, exports every symbol include/spdinv.h declares,
and rejects bad arguments synchronously (no GPU needed)."""
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
