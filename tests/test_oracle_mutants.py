"""Pins the pins: plants one plausible mistake at a time in a temporary copy
of the oracle (dropped term, off-by-one bound, transposed operand, wrong
sign) and checks that the closed-form and LAPACK checks reject every mutant;
the same for copies of its Python error measures and backward against their
hand-derived values.  CPU only; the committed oracle is never modified."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from oracle import closed_forms as cf
import spd_inputs as si

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTANTS = {
    "potf2_pivot_bound": ("for (int64_t k = 0; k < j; ++k) d -=", "for (int64_t k = 0; k + 1 < j; ++k) d -="),
    "potf2_transposed": ("s -= AT(A, i, k) * AT(A, j, k);", "s -= AT(A, i, k) * AT(A, k, j);"),
    "potf2_no_divide": ("AT(A, i, j) = s / ljj;", "AT(A, i, j) = s;"),
    "trti2_k_bound": ("for (int64_t k = j + 1; k <= i; ++k)", "for (int64_t k = j + 1; k < i; ++k)"),
    "trti2_sign": ("col[i] = -s * xjj;", "col[i] = s * xjj;"),
    "lauu2_drop_diag": ("for (int64_t k = i; k < n; ++k)", "for (int64_t k = i + 1; k < n; ++k)"),
    "lauu2_transposed": ("s += AT(A, k, i) * AT(A, k, j);", "s += AT(A, i, k) * AT(A, k, j);"),
}


def _pins_pass(lib):
    f = lib.oracle_potri
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
    f.restype = ctypes.c_int

    def potri(A):
        M = np.array(A, dtype=np.float64, order="F", copy=True)
        info = f(M.shape[0], M.ctypes.data, M.shape[0])
        Lo = np.tril(M)
        return Lo + np.tril(Lo, -1).T, info

    n = 40
    X, info = potri(si.tridiag(n))
    if info != 0 or not np.allclose(X, cf.tridiag_inverse(n), rtol=1e-10, atol=1e-12):
        return False
    A, _, _ = si.spectral_spd(64, 1e2, seed=1)
    X, info = potri(A)
    c, _ = lapack.dpotrf(A, lower=1, clean=1)
    inv, _ = lapack.dpotri(c, lower=1)
    ref = np.tril(inv) + np.tril(inv, -1).T
    return info == 0 and np.linalg.norm(X - ref) <= 1e-10 * np.linalg.norm(ref)


def _compile(src_text, tmp_path, name):
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", str(c), "-o", str(so), "-lm"])
    return ctypes.CDLL(str(so))


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_compile(open(SRC).read(), tmp_path, "orig"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    assert not _pins_pass(_compile(text.replace(old, new), tmp_path, name))


# Planted mistakes in the oracle's Python measures; each must fail its pin.
PY_MUTANTS = {
    "ratio_eps": ("lapack_ratio", "* EPS))", "* 2.0 * EPS))"),
    "ratio_order": ("lapack_ratio", "A @ X", "X @ A"),
    "ratio_norm": ("lapack_ratio", "np.linalg.norm(R, 1)", "np.linalg.norm(R, np.inf)"),
    "ratio_no_n": ("lapack_ratio", "(n * np.linalg", "(np.linalg"),
    "relF_denominator": ("rel_frobenius", "np.linalg.norm(Y))", "np.linalg.norm(X))"),
    "backward_no_sym": ("backward", "-(M + M.T) / 2.0", "-M"),
    "backward_sign": ("backward", "-(M + M.T) / 2.0", "(M + M.T) / 2.0"),
    "backward_order": ("backward", "X @ G @ X", "G @ X @ X"),
}


def _mutated(fn_name, old=None, new=None):
    """A fresh copy of an oracle function, with `old` replaced by `new`."""
    import inspect
    import textwrap

    import oracle
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fn_name)))
    if old is not None:
        assert src.count(old) == 1, (fn_name, old)
        src = src.replace(old, new)
    ns = {"np": np, "EPS": oracle.EPS}
    exec(src, ns)
    return ns[fn_name]


def _pin_for(fn_name):
    import test_oracle_pins as P
    return {"lapack_ratio": P.pin_lapack_ratio, "rel_frobenius": P.pin_rel_frobenius,
            "backward": P.pin_backward}[fn_name]


@pytest.mark.parametrize("fn_name", ["lapack_ratio", "rel_frobenius", "backward"])
def test_unmutated_measure_passes(fn_name):
    _pin_for(fn_name)(_mutated(fn_name))


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_measure_mutant_is_caught(name):
    fn_name, old, new = PY_MUTANTS[name]
    with pytest.raises(AssertionError):
        _pin_for(fn_name)(_mutated(fn_name, old, new))
