"""Pins of the periodic-search oracle (Sect. 2.3-2.4, Eq. result, App. B).

* closed forms of Eq. result: K = 1 gives Delta = Delta_1 and
  ln P = ln L_1 + ln(2)/2; equal sigma_k give the plain mean depth;
  Delta/sigma = sum(Delta_k/var_k) / sqrt(sum 1/var_k);
* each term of the second sum is -2 ln of the Gaussian-product integral of
  App. B, checked by numerical quadrature;
* interpolation is exact on linear data and drops epochs across gaps;
* with white noise and no design matrix the single events are exactly
  independent, so the fold equals one GLS fit of the full periodic template
  (the independence assumption of Sect. 2.3 holds exactly), and a noiseless
  periodic injection is recovered at its period, phase and duration;
* a brute-force loop over epochs agrees with the vectorised fold;
* the argmax takes the first maximum in duration-major, phase order.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import linear, periodic
from paper_2402_06835_gb300 import synth


def test_k1_closed_form():
    lnp, d, s = periodic.combine([3e-3], [4e-8], [7.5])
    assert d == pytest.approx(3e-3, rel=1e-15)
    assert s == pytest.approx(2e-4, rel=1e-15)
    assert lnp == pytest.approx(7.5 + 0.5 * np.log(2.0), rel=1e-15)


def test_equal_sigma_mean_depth():
    dk = np.array([1e-3, 2e-3, 4e-3, -1e-3])
    lnp, d, s = periodic.combine(dk, np.full(4, 1e-6), np.zeros(4))
    assert d == pytest.approx(dk.mean(), rel=1e-14)
    assert s == pytest.approx(np.sqrt(1e-6 / 4), rel=1e-14)


def test_snr_identity():
    rng = np.random.default_rng(4)
    dk = rng.normal(1e-3, 5e-4, 12)
    vk = rng.uniform(1e-8, 9e-8, 12)
    _, d, s = periodic.combine(dk, vk, np.zeros(12))
    num = dk / vk
    assert d / s == pytest.approx(num.sum() / np.sqrt((1 / vk).sum()), rel=1e-13)


def _gauss_product(dk, sk2, delta, s2):
    """App. B: (1/sqrt(2 pi s2)) * integral of the two Gaussian factors."""
    f = lambda x: (np.exp(-(x - dk) ** 2 / (2 * sk2))
                   * np.exp(-(x - delta) ** 2 / (2 * s2)))
    lo = min(dk, delta) - 40 * np.sqrt(max(sk2, s2))
    hi = max(dk, delta) + 40 * np.sqrt(max(sk2, s2))
    val, _ = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=400,
                            points=[dk, delta])
    return val / np.sqrt(2 * np.pi * s2)


@pytest.mark.parametrize("dk,sk2,delta,s2", [(1e-3, 4e-8, 1.5e-3, 1e-8),
                                              (-2e-3, 1e-6, 3e-4, 3e-7),
                                              (0.0, 2e-8, 0.0, 2e-8)])
def test_penalty_against_gaussian_product_integral(dk, sk2, delta, s2):
    """The depth-mismatch term is -2 ln of the App. B integral relative to its
    value at equal depths; the logarithmic terms are those of the integral's
    prefactor with the sign that Eq. result prints.  (App. B's integral gives
    +1/2 ln(sk2/(s2+sk2)) per event, while Eq. result, in Sect. 2.3 and again
    at the end of App. B, subtracts 1/2 [ln sk2 - ln(s2+sk2)]; the printed
    sign is the one kept.)"""
    I = _gauss_product(dk, sk2, delta, s2)
    I0 = _gauss_product(dk, sk2, dk, s2)          # equal depths: prefactor
    log_prefactor_sq = 2.0 * np.log(I0)           # ln(sk2 / (s2 + sk2))
    mismatch = -2.0 * np.log(I / I0)              # (dk-delta)^2/(sk2+s2)
    pen = periodic.epoch_penalty(dk, sk2, delta, s2)
    assert pen == pytest.approx(log_prefactor_sq + mismatch, rel=1e-9, abs=1e-12)
    # the derivation's own value of -2 ln I differs only in that sign
    assert -2.0 * np.log(I) == pytest.approx(-log_prefactor_sq + mismatch,
                                             rel=1e-9, abs=1e-12)


def test_interpolation_exact_on_linear_data_and_gaps():
    t0s = np.concatenate([np.arange(10) * 0.1, 2.0 + np.arange(10) * 0.1])
    a = np.stack([1.0 + 2.0 * t0s, 2.0 - t0s])                  # (n_D=2, n)
    var = np.stack([(1.0 + t0s) ** 2, (3.0 + t0s) ** 2])
    T = np.array([0.05, 0.37, 0.95, 1.5, 2.44, 2.9, 2.95])
    valid, dk, sk, lk = periodic.interpolate(t0s, a, var, a, T, dt=0.1)
    # 0.95 lies between 0.9 and 2.0 (gap), 1.5 too; 2.95 has no right node
    assert valid[0].tolist() == [True, True, False, False, True, False, False]
    ok = valid[0]
    np.testing.assert_allclose(dk[0, ok], 1.0 + 2.0 * T[ok], rtol=1e-14)
    np.testing.assert_allclose(sk[0, ok], 1.0 + T[ok], rtol=1e-14)
    np.testing.assert_allclose(dk[1, ok], 2.0 - T[ok], rtol=1e-14)
    # an epoch exactly on a node has weight 0 on the right node
    v2, d2, _, _ = periodic.interpolate(t0s, a, var, a, np.array([0.3]), dt=0.1)
    assert v2[0, 0] and d2[0, 0] == pytest.approx(1.6, rel=1e-15)


def _brute_fold(t0s, depth, var, dlnl, P, dt, d, j):
    n_phi = int(np.ceil(P / dt))
    out = []
    k = 0
    while True:
        T = t0s[0] + (j / n_phi + k) * P
        if T > t0s[-1]:
            break
        k += 1
        i = -1
        for q in range(len(t0s)):
            if t0s[q] <= T:
                i = q
        if i < 0 or i > len(t0s) - 2 or t0s[i + 1] - t0s[i] > 1.5 * dt:
            continue
        w = (T - t0s[i]) / (t0s[i + 1] - t0s[i])
        vals = []
        for arr, f in ((depth, None), (var, np.sqrt), (dlnl, None)):
            a, b = arr[d, i], arr[d, i + 1]
            if f is not None:
                a, b = f(a), f(b)
            vals.append((1 - w) * a + w * b)
        if all(np.isfinite(vals)):
            out.append(vals)
    if not out:
        return -np.inf, np.nan, np.nan
    out = np.array(out)
    return periodic.combine(out[:, 0], out[:, 1] ** 2, out[:, 2])


def test_vectorised_fold_matches_brute_force():
    rng = np.random.default_rng(8)
    t0s = np.concatenate([np.arange(60), np.arange(75, 140)]) * 0.01
    n = len(t0s)
    depth = rng.normal(0, 1e-3, (2, n))
    var = rng.uniform(1e-8, 4e-8, (2, n))
    dlnl = rng.uniform(0, 5, (2, n))
    depth[1, 40] = np.nan
    for P in [0.11, 0.237, 0.61]:
        f = periodic.fold_period(t0s, depth, var, dlnl, P, 0.01)
        for d in range(2):
            for j in range(f["n_phi"]):
                lnp, dd, ss = _brute_fold(t0s, depth, var, dlnl, P, 0.01, d, j)
                if np.isfinite(lnp):
                    assert f["lnP"][d, j] == pytest.approx(lnp, rel=1e-12)
                    assert f["depth"][d, j] == pytest.approx(dd, rel=1e-12)
                else:
                    assert f["lnP"][d, j] == -np.inf


def _white_curve(n, period_slots, depth, epoch_slot, dur_slots, seed=0,
                 noise=True):
    rng = np.random.default_rng(seed)
    t = np.arange(n) * synth.CADENCE_DAYS
    dv = np.full(n, 1e-6)
    y = rng.standard_normal(n) * 1e-3 if noise else np.zeros(n)
    for c in range(epoch_slot, n, period_slots):
        y[c:c + dur_slots] -= depth
    return t, y, dv


def test_p6_independence_exact_for_white_noise():
    n, ps = 600, 97
    t, y, dv = _white_curve(n, ps, 2e-3, 20, 8, seed=3)
    X = np.zeros((n, 0))
    D = 8 * synth.CADENCE_DAYS
    t0s = t.copy()
    res = linear.linear_search(t, y, dv, [], X, t0s, np.array([D]))
    dt = synth.CADENCE_DAYS
    P = ps * dt
    f = periodic.fold_period(t0s, res["depth"], res["var"], res["dlnl"], P, dt)
    model = linear.DenseModel(t, y, dv, [], X)
    for j in [0, 13, 24, 60]:
        epochs = [t0s[0] + (j / f["n_phi"] + k) * P for k in range(10)]
        epochs = [T for T in epochs if T <= t0s[-1]]
        # on-grid phase: every epoch is a grid node up to rounding, and the
        # fold then takes that node's single event; the joint template is
        # the union of those nodes' windows
        nodes = [int(np.rint((T - t0s[0]) / dt)) for T in epochs]
        m = sum(linear.box_template(t, t0s[q], D) for q in nodes)
        dj, vj, _ = model.fit_templates(m[:, None])
        assert f["depth"][0, j] == pytest.approx(dj[0], rel=1e-9, abs=1e-12)
        assert f["sigma"][0, j] ** 2 == pytest.approx(vj[0], rel=1e-9)


def test_p7_noiseless_periodic_injection():
    n, ps, dur = 720, 131, 9
    t, y, dv = _white_curve(n, ps, 3e-3, 40, dur, noise=False)
    X = np.zeros((n, 0))
    Ds = np.array([5, 9, 14]) * synth.CADENCE_DAYS
    res = linear.linear_search(t, y, dv, [], X, t, Ds)
    dt = synth.CADENCE_DAYS
    periods = np.array([97, 131, 150]) * dt
    out = periodic.periodic_search(t, res["depth"], res["var"], res["dlnl"],
                                   periods, dt)
    b = periodic.best(out, periods)
    assert b["period"] == pytest.approx(131 * dt)
    assert b["D_idx"] == 1
    assert b["depth"] == pytest.approx(3e-3, rel=1e-12)
    # box of 9 samples centred on t0 starts at slot 40: t0 = t[44] + dt/2
    # is not a node; the grid node with the same window is t[44]
    assert b["T0"] == pytest.approx(t[44], abs=1e-12)
    f = periodic.fold_period(t, res["depth"], res["var"], res["dlnl"],
                             131 * dt, dt)
    j = out["phase_idx"][1]
    # no penalty: all single-event depths are equal, ln P = sum gains + K/2 ln(1+1/K)... ->
    K = f["K"][1, j]
    gains = 0.5 * (3e-3) ** 2 / (1e-6 / dur)
    expect = K * gains - 0.5 * K * (np.log(1.0) - np.log(1.0 + 1.0 / K))
    assert f["lnP"][1, j] == pytest.approx(expect, rel=1e-9)


def test_argmax_first_in_duration_then_phase():
    t0s = np.arange(50) * 0.01
    depth = np.full((2, 50), 1e-3)
    var = np.full((2, 50), 1e-6)
    dlnl = np.full((2, 50), 1.0)
    out = periodic.periodic_search(t0s, depth, var, dlnl, np.array([0.1]), 0.01)
    # every cell ties: first duration, first phase
    assert out["D_idx"][0] == 0 and out["phase_idx"][0] == 0
    dlnl2 = dlnl.copy()
    dlnl2[1] += 1e-3
    out2 = periodic.periodic_search(t0s, depth, var, dlnl2, np.array([0.1]), 0.01)
    assert out2["D_idx"][0] == 1 and out2["phase_idx"][0] == 0


def test_no_valid_cell():
    t0s = np.arange(20) * 0.01
    nan = np.full((1, 20), np.nan)
    out = periodic.periodic_search(t0s, nan, nan, nan, np.array([0.05]), 0.01)
    assert out["Q"][0] == 0.0 and out["lnP"][0] == -np.inf
    assert out["D_idx"][0] == -1


def test_mask_transits_matches_nearest_transit_distance():
    """The oracle's mask (Sect. 3.3: windows of width 2 D centred on the
    detected transits) equals the brute-force minimum distance to any
    transit T0 + n P, away from ties at the window edge."""
    rng = np.random.default_rng(91)
    t0s = np.sort(rng.uniform(1000.0, 1010.0, 3000))
    g = dict(depth=rng.normal(0, 1e-3, (2, 3000)), var=rng.uniform(1e-8, 2e-8, (2, 3000)),
             dlnl=rng.uniform(0, 3, (2, 3000)))
    for P, T0, hw in ((0.37, 1000.11, 0.02), (1.9, 1003.3, 0.05), (7.0, 995.5, 0.1)):
        d, v, l, m = periodic.mask_transits(t0s, g["depth"], g["var"], g["dlnl"], P, T0, hw)
        ns = np.arange(-40, 60)
        brute = np.min(np.abs(t0s[:, None] - (T0 + ns[None, :] * P)), axis=1)
        clear = np.abs(brute - hw) > 1e-9
        assert np.array_equal(m[clear], (brute < hw)[clear])
        assert np.isnan(d[:, m]).all() and np.isnan(v[:, m]).all() and np.isnan(l[:, m]).all()
        assert np.array_equal(d[:, ~m], g["depth"][:, ~m])
        assert 0 < m.sum() < len(t0s)


def test_mask_then_search_finds_the_second_planet():
    """Multi-planet search on the oracle (Sect. 2.5): on a white-noise grid
    with two injected periodic signals the first search finds the stronger,
    and after masking its transits the second search finds the other."""
    rng = np.random.default_rng(5)
    dt = 2.0 / 1440.0
    t0s = np.arange(2400) * dt
    n = len(t0s)
    depth = rng.normal(0, 2e-4, (1, n))
    var = np.full((1, n), 4e-8)
    for P, T0, amp in ((0.41, 0.13, 2.4e-3), (0.67, 0.29, 1.6e-3)):
        ph = np.abs(((t0s - T0 + 0.5 * P) % P) - 0.5 * P)
        depth[0, ph < 0.01] += amp
    dlnl = depth ** 2 / (2 * var)
    periods = np.linspace(0.3, 0.9, 400)
    r1 = periodic.periodic_search(t0s, depth, var, dlnl, periods, dt)
    b1 = periodic.best(r1, periods)
    assert abs(b1["period"] - 0.41) < 0.005
    d2, v2, l2, _ = periodic.mask_transits(t0s, depth, var, dlnl, b1["period"], b1["T0"], 0.03)
    r2 = periodic.periodic_search(t0s, d2, v2, l2, periods, dt)
    b2 = periodic.best(r2, periods)
    assert abs(b2["period"] - 0.67) < 0.005


def test_rotation_alias_keep_worked_cases():
    """Sect. 3's criterion |dP - ceil(dP)| < 0.02 with dP = P / P_star, on cases
    worked by hand for P_star = 2 d (dP and the distance to the ceiling)."""
    P = np.array([1.99, 2.01, 3.97, 1.0, 4.0, 4.03, 0.5, 6.1, np.nan])
    # dP:        0.995 1.005 1.985  0.5  2.0  2.015 0.25 3.05
    # to ceil:   0.005 0.995 0.015  0.5  0    0.985 0.75 0.95
    want = np.array([False, True, False, True, False, True, True, True, True])
    assert np.array_equal(periodic.rotation_alias_keep(P, 2.0), want)
    # the wording's two-sided reading also drops 2.01 and 4.03 (nearest integer)
    want_sym = np.array([False, False, False, True, False, False, True, True, True])
    assert np.array_equal(periodic.rotation_alias_keep(P, 2.0, symmetric=True), want_sym)
    # the inequality is strict: tol = 0 keeps every period, exact multiples too
    assert periodic.rotation_alias_keep(P, 2.0, tol=0.0).all()
