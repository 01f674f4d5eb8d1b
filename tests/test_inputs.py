"""The seeded input generators (spd_inputs.py) produce what their docstrings
and the workload recipe state: exact symmetry, column-major order, the
prescribed spectrum and condition number, integer structure where claimed,
SPD-ness, ranges, and the same bits for the same seed."""
import numpy as np
import pytest

import spd_inputs as si


@pytest.mark.parametrize("n,cond", [(2, 10.0), (17, 1e3), (64, 1e6)])
def test_spectral_spd(n, cond):
    A, Q, lam = si.spectral_spd(n, cond, seed=si.SEED_BASE + 5)
    assert A.flags.f_contiguous and A.dtype == np.float64
    assert np.array_equal(A, A.T)
    assert lam[0] == 1.0 and lam[-1] == cond and np.all(np.diff(lam) >= 0)
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    ev = np.linalg.eigvalsh(A)
    assert np.allclose(ev, lam, rtol=1e-10 * cond, atol=0)
    assert np.linalg.cond(A) == pytest.approx(cond, rel=1e-8 * cond)


def test_spectral_spd_is_deterministic_per_seed():
    a1, _, l1 = si.spectral_spd(20, 1e4, seed=11)
    a2, _, l2 = si.spectral_spd(20, 1e4, seed=11)
    a3, _, _ = si.spectral_spd(20, 1e4, seed=12)
    assert np.array_equal(a1, a2) and np.array_equal(l1, l2)
    assert not np.array_equal(a1, a3)


def test_log_uniform_spectrum_is_log_uniform():
    lam = si.log_uniform_spectrum(20000, 1e4, seed=3)
    x = np.log10(lam[1:-1])
    assert x.min() >= 0.0 and x.max() <= 4.0
    # the four decades hold about a quarter of the values each
    counts = np.histogram(x, bins=4, range=(0, 4))[0] / x.size
    assert np.all(np.abs(counts - 0.25) < 0.02)


def test_tridiag_and_integer_bidiagonal():
    T = si.tridiag(6)
    assert T.flags.f_contiguous and np.array_equal(T, T.T)
    assert np.array_equal(np.diag(T), 2 * np.ones(6)) and np.array_equal(np.diag(T, -1), -np.ones(5))
    assert np.count_nonzero(T) == 6 + 2 * 5
    A, s = si.bidiag_integer_spd(9, seed=4)
    assert set(np.unique(s)) <= {-1, 1} and s.shape == (8,)
    Lf = np.eye(9) + np.diag(s.astype(np.float64), -1)
    assert np.array_equal(A, Lf @ Lf.T)  # A = L L^T exactly (small integers)
    assert np.array_equal(A, np.rint(A))


@pytest.mark.parametrize("n,shift", [(16, 0.1), (100, 1.0)])
def test_wishart_is_spd_above_the_shift(n, shift):
    A = si.wishart_spd(n, shift, seed=9)
    assert A.flags.f_contiguous and np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() >= shift * (1 - 1e-12)


def test_batch_sizes_cover_the_range():
    s = si.batch_sizes(4096, 16, 256, seed=si.SEED_BASE + 3)
    assert s.min() == 16 and s.max() == 256 and s.dtype == np.int64
    assert abs(s.mean() - 136) < 4  # uniform on {16..256}: mean 136
    mats = si.wishart_batch(s[:5], 0.1, seed=1)
    assert [m.shape[0] for m in mats] == list(s[:5])


def test_symmetric_gaussian_and_integer_spd3():
    G = si.symmetric_gaussian(7, seed=2)
    assert G.flags.f_contiguous and np.array_equal(G, G.T)
    for seed in range(10):
        A = si.integer_spd3(seed)
        assert A.dtype == np.int64 and np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(A.astype(np.float64)).min() >= 1 - 1e-9  # M^T M + I
