"""Pins of the ADM nonnegative completion oracle (App. A): an exact fixed point,
convergence of the fit on synthetic nonnegative low-rank data, satisfied
constraints where nonnegativity is active, and recovery of the unobserved
entries."""
import numpy as np

from oracle import adm


def _nonneg_lowrank(m, n, r, seed, zeros=0.0):
    rng = np.random.default_rng(seed)
    X = rng.random((m, r)) + 0.1
    Y = rng.random((r, n)) + 0.1
    if zeros:
        X[rng.random((m, r)) < zeros] = 0.0
        Y[rng.random((r, n)) < zeros] = 0.0
    return X, Y, X @ Y


def _sample(m, n, frac, seed):
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < frac
    rows, cols = np.nonzero(mask)
    return rows, cols, mask


def test_the_true_factors_are_a_fixed_point():
    # Z = M, U = X*, Lambda = 0: the X step solves (X* Y Y^T + alpha X*) (Y Y^T + alpha I)^-1
    # = X*, and likewise Y; a dropped proximal term or a wrong Z breaks it.
    X, Y, M = _nonneg_lowrank(40, 30, 4, 1)
    rows, cols, _ = _sample(40, 30, 0.35, 2)
    st = {}
    Xk, Yk = adm.complete_slice_adm(rows, cols, M[rows, cols], 40, 30, 4, 25, 0.3, 1.0, seed=5, s=0,
                                    X0=X, Y0=Y.T, state=st)
    assert np.allclose(Xk, X, atol=1e-9) and np.allclose(Yk, Y.T, atol=1e-9)
    assert np.allclose(st["U"], X, atol=1e-9) and np.abs(st["Lam"]).max() < 1e-9


def test_fit_on_the_observed_entries_converges():
    X, Y, M = _nonneg_lowrank(60, 45, 3, 3)
    rows, cols, _ = _sample(60, 45, 0.4, 4)
    hist = []
    adm.complete_slice_adm(rows, cols, M[rows, cols], 60, 45, 3, 1500, 0.3, 1.0, seed=7, s=1, history=hist)
    norm = np.linalg.norm(M[rows, cols])
    assert hist[0] > 0.1 * norm
    assert hist[49] < 0.1 * norm       # the fast first phase
    assert hist[-1] < 1e-9 * norm      # and, more slowly, the exact fit


def test_constraints_hold_where_nonnegativity_is_active():
    # factors with exact zeros: the nonnegative solution lies on the boundary, where
    # U = max(0, .) and the multipliers do the work; a wrong multiplier sign leaves
    # X far from U or the fit far from zero.
    X, Y, M = _nonneg_lowrank(50, 40, 3, 8, zeros=0.3)
    rows, cols, _ = _sample(50, 40, 0.6, 9)
    st, hist = {}, []
    Xk, Yk = adm.complete_slice_adm(rows, cols, M[rows, cols], 50, 40, 3, 1500, 0.3, 1.0, seed=3, s=4,
                                    history=hist, state=st)
    scale = np.abs(Xk).max()
    assert st["U"].min() >= 0.0 and st["VT"].min() >= 0.0
    assert np.abs(Xk - st["U"]).max() < 1e-6 * scale
    assert np.abs(Yk - st["VT"]).max() < 1e-6 * np.abs(Yk).max()
    assert hist[-1] < 1e-5 * np.linalg.norm(M[rows, cols])


def test_recovery_of_unobserved_entries():
    X, Y, M = _nonneg_lowrank(60, 45, 3, 5)
    rows, cols, mask = _sample(60, 45, 0.4, 6)
    Xa, Ya = adm.complete_slice_adm(rows, cols, M[rows, cols], 60, 45, 3, 1500, 0.3, 1.0, seed=9, s=2)
    hidden = ~mask
    err = np.linalg.norm((Xa @ Ya.T - M)[hidden]) / np.linalg.norm(M[hidden])
    assert err < 1e-3


def test_seeded_start_is_positive_and_deterministic():
    a = adm.init_x(11, 3, 20, 4, 2.0)
    assert a.shape == (20, 4) and np.array_equal(a, adm.init_x(11, 3, 20, 4, 2.0))
    lo, hi = np.sqrt(2.0 / 4) * 0.5, np.sqrt(2.0 / 4) * 1.5
    assert a.min() >= lo and a.max() < hi and not np.array_equal(a, adm.init_x(11, 4, 20, 4, 2.0))


def test_no_observed_entries_gives_zero_factors():
    Xk, Yk = adm.complete_slice_adm(np.zeros(0, int), np.zeros(0, int), np.zeros(0), 5, 4, 2, 3, 0.3, 1.0, 1, 0)
    assert not Xk.any() and not Yk.any()
