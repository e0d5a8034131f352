"""Pins of the exact periodic-template oracle (Sect. 2.4's Q(P) read as one
fit of Eq. ls with a periodic transit column, Sect. 2.3's independence
approximation).

* brute force: the periodic template against a per-sample loop over every
  transit index in a wide range;
* closed-form count: on a dyadic regular grid every full window holds
  exactly D/dt samples;
* reduction: a period longer than the data leaves one transit, and the fit
  is the linear search's at (T0, D);
* white-noise closed form: with Sigma diagonal and X = [1] the fit is the
  two-parameter weighted regression (Cramer's rule);
* Eq. result is exact without correlations: with Sigma diagonal and no X
  columns, the single events at T0 + n P combined with Eq. result give the
  same depth and variance as the exact fit (a dropped or extra window
  breaks this);
* exact recovery: noiseless y = X w + Delta m_P gives Delta back under a
  correlated covariance;
* the semiseparable reference agrees with the dense one on periodic
  templates.
"""
import math

import numpy as np
import pytest

from oracle import linear, periodic, refine, semisep
from paper_2402_06835_gb300 import synth


def test_periodic_template_brute_force():
    rng = np.random.default_rng(5)
    t = np.sort(rng.uniform(100.0, 105.0, 60))
    for kind in ("box", "trapezoid"):
        for P, T0, D in ((0.7, 101.13, 0.2), (0.45, 96.0, 0.225), (3.0, 104.9, 0.5)):
            m = refine.periodic_template(t, P, T0, D, kind, 0.25)
            want = np.zeros_like(t)
            for a, ta in enumerate(t):
                for n in range(-400, 400):
                    c = T0 + float(n) * P
                    if c - D * 0.5 <= ta < c + D * 0.5:
                        if kind == "box":
                            want[a] += -1.0
                        else:
                            want[a] += -min(max((D * 0.5 - abs(ta - c)) / (0.25 * D), 0.0), 1.0)
            assert np.array_equal(m, want)


def test_periodic_template_window_count_on_dyadic_grid():
    dt = 1.0 / 64.0
    t = np.arange(4000) * dt                       # exact in binary
    P, D, T0 = 3.0, 5.0 * dt, 0.5 * dt + 1.0      # centres half a cadence off the grid
    m = refine.periodic_template(t, P, T0, D)
    n_full = sum(1 for n in range(-10, 40)
                 if T0 + n * P - D / 2 >= t[0] and T0 + n * P + D / 2 <= t[-1])
    assert n_full == math.floor((t[-1] - T0 - D / 2) / P) + 1
    assert int(-m.sum()) == 5 * n_full
    assert set(np.unique(m)) == {0.0, -1.0}


def test_single_transit_is_the_linear_search():
    lc = synth.small_curve(n=400, seed=11)
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    span = lc.t[-1] - lc.t[0]
    T0, D = lc.t[137], 0.06
    r = refine.refine(model, [(10.0 * span, T0, D)])
    ls = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, [T0], [D], model=model)
    assert r["depth"][0] == ls["depth"][0, 0]
    assert r["var"][0] == ls["var"][0, 0]
    assert r["dlnl"][0] == ls["dlnl"][0, 0]


def test_white_noise_two_parameter_regression():
    rng = np.random.default_rng(8)
    n = 700
    t = np.sort(rng.uniform(0.0, 6.0, n))
    dv = rng.uniform(0.5e-6, 2e-6, n)
    y = rng.normal(0, 1e-3, n) + 1.0
    P, T0, D = 0.83, 0.31, 0.09
    y = y - 2e-3 * (refine.periodic_template(t, P, T0, D) != 0)
    model = linear.DenseModel(t, y, dv, [], np.ones((n, 1)))
    r = refine.refine(model, [(P, T0, D)])
    m = refine.periodic_template(t, P, T0, D)
    w = 1.0 / dv
    Sw, Sm, Smm = w.sum(), (w * m).sum(), (w * m * m).sum()
    Sy, Smy = (w * y).sum(), (w * m * y).sum()
    det = Sw * Smm - Sm * Sm
    depth = (Sw * Smy - Sm * Sy) / det
    var = Sw / det
    assert abs(r["depth"][0] - depth) <= 1e-10 * abs(depth)
    assert abs(r["var"][0] - var) <= 1e-10 * var
    assert abs(r["dlnl"][0] - depth * depth / (2 * var)) <= 1e-9 * r["dlnl"][0]
    assert abs(r["snr"][0] - depth / math.sqrt(var)) <= 1e-10 * r["snr"][0]
    assert abs(depth - 2e-3) < 3e-4


@pytest.mark.parametrize("kind", ["box", "trapezoid"])
def test_eq_result_is_exact_for_white_noise(kind):
    """Without correlations and shared columns the single transits are
    independent, so Eq. result's common depth and variance are the exact
    fit's; the periodic template must hold exactly the fold's windows."""
    rng = np.random.default_rng(9)
    n = 900
    t = np.sort(rng.uniform(10.0, 17.0, n))
    dv = rng.uniform(0.5e-6, 2e-6, n)
    y = rng.normal(0, 1e-3, n)
    model = linear.DenseModel(t, y, dv, [], np.zeros((n, 0)))
    for P, T0, D in ((0.61, 10.2, 0.1), (1.7, 16.95, 0.3), (0.35, 8.0, 0.05)):
        r = refine.refine(model, [(P, T0, D)], kind, 0.2)
        ns = range(math.floor((t[0] - T0) / P) - 1, math.ceil((t[-1] - T0) / P) + 2)
        epochs = np.array([T0 + float(k) * P for k in ns])
        ls = linear.linear_search(t, y, dv, [], np.zeros((n, 0)), epochs, [D], kind, 0.2,
                                  model=model)
        ok = np.isfinite(ls["depth"][0])
        _, delta, sigma = periodic.combine(ls["depth"][0, ok], ls["var"][0, ok],
                                           ls["dlnl"][0, ok])
        assert ok.sum() >= 3
        assert abs(r["depth"][0] - delta) <= 1e-10 * np.sqrt(r["var"][0])
        assert abs(r["var"][0] - sigma ** 2) <= 1e-10 * sigma ** 2


def test_noiseless_recovery_under_correlated_noise():
    lc = synth.small_curve(n=500, seed=13, p_rot=0.9, inject=None)
    P, T0, D, depth = 0.37, lc.t[40], 0.05, 2.5e-3
    w = np.array([1.0, -3e-4, 2e-4])[: lc.X.shape[1]]
    y = lc.X @ w + depth * refine.periodic_template(lc.t, P, T0, D)
    model = linear.DenseModel(lc.t, y, lc.diag_var, lc.terms, lc.X)
    r = refine.refine(model, [(P, T0, D)])
    assert abs(r["depth"][0] - depth) <= 1e-9 * depth
    assert abs(r["dlnl"][0] - 0.5 * depth * depth / r["var"][0]) <= 1e-8 * r["dlnl"][0]


def test_semisep_matches_dense():
    lc = synth.small_curve(n=600, seed=4, p_rot=1.1)
    dense = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    ss = semisep.Semisep(lc.t, lc.diag_var, lc.terms)
    cands = [(0.31, lc.t[10], 1.0 / 24.0), (0.77, lc.t[300], 0.07), (0.2, lc.t[0], 0.03)]
    a = refine.refine(dense, cands)
    b = refine.refine(ss, cands, X=lc.X, y=lc.y)
    for k in ("depth", "var", "dlnl", "snr"):
        assert np.allclose(a[k], b[k], rtol=1e-9, atol=0)


def test_invalid_candidates_are_nan():
    lc = synth.small_curve(n=200, seed=2)
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    bad = [(float("nan"), lc.t[5], 0.05), (0.3, float("inf"), 0.05), (0.3, lc.t[5], 0.0),
           (0.09, lc.t[5], 0.05), (1e6, lc.t[0] + 5e5, 0.05)]
    r = refine.refine(model, bad + [(0.3, lc.t[5], 0.05)])
    for k in ("depth", "var", "dlnl", "snr"):
        assert np.all(np.isnan(r[k][:-1]))
        assert np.isfinite(r[k][-1])
    with pytest.raises(ValueError):
        refine.periodic_template(lc.t, 0.09, lc.t[5], 0.05)
