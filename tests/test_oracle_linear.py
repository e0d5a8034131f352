"""Pins of the linear-search oracle (Sect. 2.2, Eq. ls, Eq. linear_search_ll).

* brute force: a separately coded explicit-inverse normal-equation solve in
  extended precision (numpy longdouble: 80-bit on x86-64, binary128 on
  aarch64) on tiny inputs;
* white-noise limit: with Sigma diagonal and X = [1] the GLS depth is the
  difference of the inverse-variance weighted means out of and in the window
  and its variance 1/W_in + 1/W_out (the weighted box-least-squares closed
  form, Kovacs et al. 2002), and for any template the two-parameter weighted
  regression closed form holds;
* exact recovery: noiseless y = X w* + Delta* m(t0*, D*) gives Delta* back
  under any covariance, with zero residual;
* template and window conventions (half-open window, ramp shape).
"""
import numpy as np
import pytest

from oracle import gp, linear
from paper_2402_06835_gb300 import synth


def rel_err(a, b, scale):
    return np.abs(a - b) / np.maximum(np.abs(scale), 1e-300)


# ---------------------------------------------------------------- brute force
def _ld_inverse(A):
    """Gauss-Jordan inverse with partial pivoting in numpy longdouble."""
    n = A.shape[0]
    M = np.concatenate([A.astype(np.longdouble),
                        np.eye(n, dtype=np.longdouble)], axis=1)
    for c in range(n):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if p != c:
            M[[c, p]] = M[[p, c]]
        M[c] = M[c] / M[c, c]
        col = M[:, c].copy()
        col[c] = 0
        M -= col[:, None] * M[c][None, :]
    return M[:, n:]


def _brute_force(Sigma, X, y, m):
    S = Sigma.astype(np.longdouble)
    Si = _ld_inverse(S)
    Xp = np.concatenate([X, m[:, None]], axis=1).astype(np.longdouble)
    yl = y.astype(np.longdouble)
    G = Xp.T @ Si @ Xp
    Gi = _ld_inverse(G)
    w = Gi @ (Xp.T @ Si @ yl)
    r = yl - Xp @ w
    chi2 = r @ Si @ r
    # null model
    X0 = X.astype(np.longdouble)
    G0i = _ld_inverse(X0.T @ Si @ X0)
    w0 = G0i @ (X0.T @ Si @ yl)
    r0 = yl - X0 @ w0
    chi2_0 = r0 @ Si @ r0
    return float(w[-1]), float(Gi[-1, -1]), float(0.5 * (chi2_0 - chi2))


@pytest.mark.parametrize("kind", ["box", "trapezoid", "limb_quad"])
def test_p1_brute_force_tiny(kind):
    lc = synth.small_curve(n=48, seed=3, p_rot=0.2)
    t, y, dv = lc.t, lc.y, lc.diag_var
    terms = lc.terms + [(gp.EXP, (2e-3, 0.05))]
    Sigma = gp.covariance(t, dv, terms)
    t0s = t[[5, 20, 33, 46]]
    Ds = np.array([0.02, 0.05])
    res = linear.linear_search(t, y, dv, terms, lc.X, t0s, Ds, kind=kind,
                               ingress_frac=0.2)
    for j, D in enumerate(Ds):
        for i, t0 in enumerate(t0s):
            m = linear.template(t, t0, D, kind, 0.2)
            d, v, l = _brute_force(Sigma, lc.X, y, m)
            sd = np.sqrt(v)
            assert rel_err(res["depth"][j, i], d, max(abs(d), sd)) < 1e-12
            assert rel_err(res["var"][j, i], v, v) < 1e-12
            assert rel_err(res["dlnl"][j, i], l, max(l, 1.0)) < 1e-12


# ------------------------------------------------------ white-noise closed form
def test_p2_white_noise_box_is_weighted_bls():
    rng = np.random.default_rng(11)
    n = 400
    t = np.arange(n) * synth.CADENCE_DAYS
    dv = rng.uniform(0.5e-6, 3e-6, n)
    y = 1.0 + rng.standard_normal(n) * np.sqrt(dv)
    X = np.ones((n, 1))
    t0s = t[[0, 37, 150, 399]]
    Ds = np.array([0.01, 0.05, 0.11])
    res = linear.linear_search(t, y, dv, [], X, t0s, Ds)
    for j, D in enumerate(Ds):
        for i, t0 in enumerate(t0s):
            inside = (t >= t0 - D / 2) & (t < t0 + D / 2)
            w = 1.0 / dv
            W_in, W_out = w[inside].sum(), w[~inside].sum()
            m_in = (w[inside] * y[inside]).sum() / W_in
            m_out = (w[~inside] * y[~inside]).sum() / W_out
            depth = m_out - m_in
            var = 1.0 / W_in + 1.0 / W_out
            assert res["depth"][j, i] == pytest.approx(depth, rel=1e-10, abs=1e-12)
            assert res["var"][j, i] == pytest.approx(var, rel=1e-12)
            assert res["dlnl"][j, i] == pytest.approx(0.5 * depth ** 2 / var,
                                                      rel=1e-8, abs=1e-10)


def test_p2_white_noise_trapezoid_two_parameter_regression():
    rng = np.random.default_rng(12)
    n = 300
    t = np.arange(n) * synth.CADENCE_DAYS
    dv = rng.uniform(0.5e-6, 3e-6, n)
    y = 1.0 + rng.standard_normal(n) * np.sqrt(dv)
    res = linear.linear_search(t, y, dv, [], np.ones((n, 1)), t[[50, 200]],
                               np.array([0.07]), kind="trapezoid",
                               ingress_frac=0.25)
    for i, t0 in enumerate(t[[50, 200]]):
        m = linear.trapezoid_template(t, t0, 0.07, 0.25)
        w = 1.0 / dv
        Sw, Sm, Smm = w.sum(), (w * m).sum(), (w * m * m).sum()
        Sy, Smy = (w * y).sum(), (w * m * y).sum()
        det = Sw * Smm - Sm * Sm
        depth = (Sw * Smy - Sm * Sy) / det
        var = Sw / det
        assert res["depth"][0, i] == pytest.approx(depth, rel=1e-9)
        assert res["var"][0, i] == pytest.approx(var, rel=1e-11)


def test_white_noise_logdet_and_null():
    dv = np.array([1e-6, 2e-6, 4e-6, 3e-6])
    t = np.arange(4.0)
    y = np.array([1.0, 2.0, 0.5, 1.5])
    model = linear.DenseModel(t, y, dv, [], np.zeros((4, 0)))
    assert model.logdet == pytest.approx(np.sum(np.log(dv)), rel=1e-14)
    assert model.chi2_null == pytest.approx(np.sum(y * y / dv), rel=1e-14)
    # two correlated points: |Sigma| = a^2 - c^2
    S = gp.covariance(np.array([0.0, 0.1]), np.array([1.0, 1.0]),
                      [(gp.EXP, (1.0, 0.2))])
    m2 = linear.DenseModel(np.array([0.0, 0.1]), np.zeros(2), np.ones(2),
                           [(gp.EXP, (1.0, 0.2))], np.zeros((2, 0)))
    assert m2.logdet == pytest.approx(np.log(S[0, 0] ** 2 - S[0, 1] ** 2),
                                      rel=1e-14)


# ---------------------------------------------------------- noiseless recovery
@pytest.mark.parametrize("kind", ["box", "trapezoid", "limb_quad"])
def test_p3_noiseless_recovery(kind):
    lc = synth.small_curve(n=240, seed=5, gap=30)
    t = lc.t
    t0, D, depth = t[110], 0.06, 2.5e-3
    m = linear.template(t, t0, D, kind, 0.1)
    y = lc.X @ np.array([1.0, -3e-3]) + depth * m
    res = linear.linear_search(t, y, lc.diag_var, lc.terms, lc.X,
                               np.array([t0]), np.array([D]), kind=kind)
    assert res["depth"][0, 0] == pytest.approx(depth, rel=1e-10)
    v = res["var"][0, 0]
    assert np.isfinite(v) and v > 0
    # the full model leaves no residual: lnL = -1/2 ln|Sigma| - N/2 ln 2 pi
    lnl = res["dlnl"][0, 0] + res["lnL_null"]
    expect = -0.5 * res["logdet"] - 0.5 * len(t) * np.log(2 * np.pi)
    assert lnl == pytest.approx(expect, rel=1e-12)
    assert res["dlnl"][0, 0] == pytest.approx(0.5 * depth ** 2 / v, rel=1e-8)


def test_gain_equals_half_depth_squared_over_var():
    """Eq. linear_search_ll at the GLS optimum: the gain over the null model
    is Delta^2 / (2 var) (a property of the least-squares projection)."""
    lc = synth.small_curve(n=200, seed=9)
    res = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X,
                               lc.t[::17], np.array([0.02, 0.05]))
    g = 0.5 * res["depth"] ** 2 / res["var"]
    np.testing.assert_allclose(res["dlnl"], g, rtol=1e-7, atol=1e-9)


def test_cholesky_solves_sigma():
    lc = synth.small_curve(n=150, seed=2)
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    S = gp.covariance(lc.t, lc.diag_var, lc.terms)
    from scipy.linalg import solve_triangular
    x = solve_triangular(model.C.T, model.yw, lower=False)    # Sigma^-1 y
    np.testing.assert_allclose(S @ x, lc.y, rtol=1e-12)


# ------------------------------------------------------------- conventions
def test_box_window_half_open_and_counts():
    t = np.arange(100) * 0.01
    m = linear.box_template(t, 0.5, 0.2)
    # t0 - D/2 = 0.4 is inside, t0 + D/2 = 0.6 is outside
    idx = np.nonzero(m)[0]
    assert np.all(m[idx] == -1.0)
    assert t[idx[0]] == pytest.approx(0.4) and t[idx[-1]] == pytest.approx(0.59)
    assert len(idx) == 20


def test_trapezoid_shape():
    t = np.linspace(-1, 1, 2001)
    m = linear.trapezoid_template(t, 0.0, 1.0, 0.2)
    assert m[np.argmin(np.abs(t))] == -1.0
    assert np.all(m[np.abs(t) >= 0.5] == 0.0)
    # ramp: halfway through ingress the template is -1/2
    assert m[np.argmin(np.abs(t + 0.4))] == pytest.approx(-0.5, abs=1e-9)
    assert np.all(m[np.abs(t) <= 0.3] == -1.0)


def test_limb_quad_shape_and_integral():
    """Centre -1, limb -(1 - u1 - u2), zero outside; no darkening is the box;
    and the area of the dip is the closed form of the quadratic law's chord
    integral, int_{-1}^{1} I(sqrt(1 - x^2)) dx = 2 - u1 (2 - pi/2) - u2 (10/3 - pi)."""
    u1, u2 = 0.45, 0.2
    D = 1.0
    t = (np.arange(2_000_001) - 1_000_000) * 1e-6          # step 1e-6, t0 = 0
    m = linear.limb_quad_template(t, 0.0, D, u1, u2)
    assert m[1_000_000] == -1.0
    assert m[np.argmin(np.abs(t + 0.5))] == pytest.approx(-(1.0 - u1 - u2), rel=1e-15)
    assert np.all(m[np.abs(t) > 0.5] == 0.0) and m[np.argmin(np.abs(t - 0.5))] == 0.0
    assert np.array_equal(linear.limb_quad_template(t, 0.0, D, 0.0, 0.0),
                          linear.box_template(t, 0.0, D))
    area = -m.sum() * 1e-6
    exact = 0.5 * D * (2.0 - u1 * (2.0 - np.pi / 2) - u2 * (10.0 / 3.0 - np.pi))
    assert area == pytest.approx(exact, rel=1e-6)
    # monotone from the limb to the centre for a physical law
    left = m[(t >= -0.5) & (t <= 0.0)]
    assert np.all(np.diff(left) <= 0.0)


def test_empty_window_gives_nan():
    lc = synth.small_curve(n=100, seed=1, gap=50)
    gap_mid = 0.5 * (lc.t[49] + lc.t[50])
    res = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X,
                               np.array([gap_mid]), np.array([0.01]))
    assert np.isnan(res["depth"][0, 0]) and np.isnan(res["var"][0, 0])
    assert np.isnan(res["dlnl"][0, 0])


# --------------------------------------- whole-grid route (explicit Sigma^-1)
def test_box_grid_brute_force_tiny():
    """The block-elimination route against the extended-precision brute force."""
    lc = synth.small_curve(n=48, seed=3, p_rot=0.2)
    t, y, dv = lc.t, lc.y, lc.diag_var
    terms = lc.terms + [(gp.EXP, (2e-3, 0.05))]
    Sigma = gp.covariance(t, dv, terms)
    t0s = t[[0, 5, 20, 33, 46, 47]]
    Ds = np.array([0.003, 0.02, 0.05])
    model = linear.DenseModel(t, y, dv, terms, lc.X)
    res = linear.box_grid(model, t0s, Ds)
    for j, D in enumerate(Ds):
        for i, t0 in enumerate(t0s):
            m = linear.box_template(t, t0, D)
            d, v, l = _brute_force(Sigma, lc.X, y, m)
            sd = np.sqrt(v)
            assert rel_err(res["depth"][j, i], d, max(abs(d), sd)) < 1e-12
            assert rel_err(res["var"][j, i], v, v) < 1e-12
            assert rel_err(res["dlnl"][j, i], l, max(l, 1.0)) < 1e-12


def test_box_grid_white_noise_is_weighted_bls():
    rng = np.random.default_rng(13)
    n = 500
    t = np.arange(n) * synth.CADENCE_DAYS
    dv = rng.uniform(0.5e-6, 3e-6, n)
    y = 1.0 + rng.standard_normal(n) * np.sqrt(dv)
    X = np.ones((n, 1))
    Ds = np.array([0.01, 0.05, 0.11])
    res = linear.box_grid(linear.DenseModel(t, y, dv, [], X), t, Ds)
    w = 1.0 / dv
    for j, D in enumerate(Ds):
        for i in (0, 1, 37, 150, 250, 498, 499):
            t0 = t[i]
            inside = (t >= t0 - D / 2) & (t < t0 + D / 2)
            W_in, W_out = w[inside].sum(), w[~inside].sum()
            depth = ((w[~inside] * y[~inside]).sum() / W_out
                     - (w[inside] * y[inside]).sum() / W_in)
            var = 1.0 / W_in + 1.0 / W_out
            assert res["depth"][j, i] == pytest.approx(depth, rel=1e-10, abs=1e-12)
            assert res["var"][j, i] == pytest.approx(var, rel=1e-12)
            assert res["dlnl"][j, i] == pytest.approx(0.5 * depth ** 2 / var,
                                                      rel=1e-8, abs=1e-10)


def test_box_grid_noiseless_recovery():
    """y = X w* + Delta* m(t0*, D*) exactly: the grid's cell at (t0*, D*)
    returns Delta* under a correlated covariance."""
    lc = synth.small_curve(n=300, seed=5, gap=30)
    t = lc.t
    t0, D, delta = t[77], 0.05, 2.5e-3
    y = lc.X @ np.array([1.0, -3e-3]) + delta * linear.box_template(t, t0, D)
    model = linear.DenseModel(t, y, lc.diag_var, lc.terms, lc.X)
    res = linear.box_grid(model, t[[76, 77, 78]], np.array([D]))
    assert res["depth"][0, 1] == pytest.approx(delta, rel=1e-12)
    assert np.isfinite(res["var"][0]).all()


@pytest.mark.parametrize("case", ["rotation", "rotation+exp", "sho_overdamped", "white"])
@pytest.mark.parametrize("design", [True, False])
def test_box_grid_matches_qr_route(case, design):
    """Both dense routes (QR of every whitened template; block elimination
    with the explicit inverse) on a gapped curve, epochs in the gap and
    beyond both ends included."""
    lc = synth.small_curve(n=360, seed=21, gap=40, design=design)
    terms = {"rotation": lc.terms,
             "rotation+exp": lc.terms + [(gp.EXP, (2e-3, 0.08))],
             "sho_overdamped": [(gp.SHO, (5e-3, 30.0, 0.3))],
             "white": []}[case]
    X = lc.X if design else np.zeros((len(lc.t), 0))
    Ds = np.array([0.004, 0.035, 0.09])
    t0s = np.concatenate([lc.t, [0.5 * (lc.t[179] + lc.t[180]), lc.t[0] - 0.01,
                                 lc.t[-1] + 0.02]])
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, terms, X)
    g = linear.box_grid(model, t0s, Ds)
    o = linear.linear_search(lc.t, lc.y, lc.diag_var, terms, X, t0s, Ds, model=model)
    for a, b in ((g["depth"], o["depth"]), (g["var"], o["var"]), (g["dlnl"], o["dlnl"])):
        assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(o["depth"])
    so = np.sqrt(o["var"][ok])
    assert np.max(rel_err(g["depth"][ok], o["depth"][ok], np.maximum(np.abs(o["depth"][ok]), so))) < 1e-11
    assert np.max(rel_err(g["var"][ok], o["var"][ok], o["var"][ok])) < 1e-11
    assert np.max(rel_err(g["dlnl"][ok], o["dlnl"][ok], np.maximum(o["dlnl"][ok], 1.0))) < 1e-10
