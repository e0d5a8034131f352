"""GPU parity of nu_mask_transits (the masking step of the multi-planet
search, Sect. 2.5 and Sect. 3.3) and of a second search after masking."""
import numpy as np
import pytest

from oracle import linear, periodic
from paper_2402_06835_gb300 import synth
from parity import FP64_TOL, periodic_compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def cu(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mask_is_bit_exact(precision):
    """Which entries are masked is decided in FP64 on both sides: the NaN
    pattern must be identical, and unmasked values untouched."""
    rng = np.random.default_rng(12)
    n = 5000
    t0s = np.sort(1500.0 + rng.uniform(0, 9.0, n))
    dty, ndt = (torch.float64, np.float64) if precision == "fp64" else (torch.float32, np.float32)
    g = {k: rng.normal(0, 1, (3, n)).astype(ndt) for k in ("depth", "var", "dlnl")}
    for P, T0, hw in ((0.37, 1500.11, 0.02), (1.9, 1503.3, 0.05), (7.0, 1495.5, 0.1),
                      (0.05, 1500.0, 0.01)):
        arrs = [cu(g[k], dty) for k in ("depth", "var", "dlnl")]
        api.nu_mask_transits(cu(t0s), *arrs, P, T0, hw, precision=precision)
        got = [a.cpu().numpy() for a in arrs]
        d, v, l, m = periodic.mask_transits(t0s, g["depth"], g["var"], g["dlnl"], P, T0, hw)
        for a, b in zip(got, (d, v, l)):
            assert np.array_equal(np.isnan(a), np.isnan(b))
            assert np.array_equal(a[~np.isnan(b)], b[~np.isnan(b)])
        assert 0 < m.sum() < n


def test_mask_rejects_bad_arguments():
    t0s = cu(np.arange(10.0))
    z = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(api.NuanceError):
        api.nu_mask_transits(t0s, z, z.clone(), z.clone(), -1.0, 0.0, 0.1)
    with pytest.raises(api.NuanceError):
        api.nu_mask_transits(t0s, z, z.clone(), z.clone(), 1.0, float("nan"), 0.1)


def test_second_planet_after_masking():
    """Two planets in a correlated-noise light curve: each side (GPU and
    oracle) searches, masks its own detection with half-width D and
    searches again; the second periodograms agree and find planet b."""
    lc = synth.small_curve(n=2200, seed=3, p_rot=1.3, sigma=4e-3, sigma_w=1e-3,
                           inject=(3e-3, 1.0 / 24.0, 0.41))
    y = synth._inject_box(lc.t, lc.y.copy(), 2.2e-3, 1.0 / 24.0, 0.67, lc.t[0] + 0.29)
    Ds = np.array([0.03, 1.0 / 24.0, 0.055])
    periods = np.linspace(0.3, 0.9, 500)
    dt = periodic.median_spacing(lc.t)
    ora = linear.linear_search(lc.t, y, lc.diag_var, lc.terms, lc.X, lc.t, Ds)
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(y))
    d, v, l = api.nu_linear_search(f, cu(lc.t), Ds)
    # first search, each side
    r1o = periodic.periodic_search(lc.t, ora["depth"], ora["var"], ora["dlnl"], periods, dt)
    b1 = periodic.best(r1o, periods)
    p1o = int(np.argmax(np.where(np.isfinite(r1o["Q"]), r1o["Q"], -np.inf)))
    r1g = api.nu_periodic_search(cu(lc.t), Ds, d, v, l, cu(periods), phase_step=dt)
    Qg = r1g["Q"].cpu().numpy()
    p1g = int(np.argmax(np.where(np.isfinite(Qg), Qg, -np.inf)))
    assert p1g == p1o and abs(periods[p1g] - 0.41) < 0.01
    # mask, each with its own detection
    Dg = float(Ds[int(r1g["D_idx"][p1g])])
    api.nu_mask_transits(cu(lc.t), d, v, l, float(periods[p1g]), float(r1g["T0"][p1g]), Dg)
    Do = float(Ds[int(r1o["D_idx"][p1o])])
    md, mv, ml, _ = periodic.mask_transits(lc.t, ora["depth"], ora["var"], ora["dlnl"],
                                           b1["period"], b1["T0"], Do)
    r2o = periodic.periodic_search(lc.t, md, mv, ml, periods, dt)
    r2g = api.nu_periodic_search(cu(lc.t), Ds, d, v, l, cu(periods), phase_step=dt)
    gpu = {k: t.cpu().numpy() for k, t in r2g.items()}
    wl, wq, differ = periodic_compare(gpu, r2o, lc.t, md, mv, ml, periods, dt, FP64_TOL,
                                      FP64_TOL, periodic.fold_period)
    b2 = periodic.best(r2o, periods)
    print(f"after masking: lnP err {wl:.2e}, Q err {wq:.2e}, ties {differ}, "
          f"second planet at {b2['period']:.4f}")
    assert abs(b2["period"] - 0.67) < 0.01


def test_per_sector_factors_with_one_fold():
    """The paper's multi-sector mode (Sect. 3.3): each sector gets its own GP
    factor and linear search, and one periodic search runs over the
    concatenated (t0, D) grids.  Both sides do the same; the periodograms
    agree and the common planet is found."""
    P, dur = 0.53, 1.0 / 24.0
    A = synth.small_curve(n=1500, seed=11, p_rot=0.9, sigma=3e-3, inject=(2.5e-3, dur, P))
    B = synth.small_curve(n=1500, seed=12, p_rot=1.4, sigma=5e-3, inject=None)
    tB = B.t + 6.0
    yB = synth._inject_box(tB, B.y.copy(), 2.5e-3, dur, P, A.injected["epoch"])
    XB = np.stack([np.ones_like(tB), tB], axis=1)
    sectors = [(A.t, A.y, A.diag_var, A.terms, A.X), (tB, yB, B.diag_var, B.terms, XB)]
    Ds = np.array([0.03, dur, 0.055])
    periods = np.linspace(0.3, 1.2, 400)
    grids_o, grids_g = [], []
    for t, y, dv, terms, X in sectors:
        grids_o.append(linear.linear_search(t, y, dv, terms, X, t, Ds))
        f = api.nu_gp_factor(cu(t), cu(dv), terms, cu(X), cu(y))
        grids_g.append(api.nu_linear_search(f, cu(t), Ds))
    t0s = np.concatenate([s[0] for s in sectors])
    go = {k: np.concatenate([g[k] for g in grids_o], axis=1) for k in ("depth", "var", "dlnl")}
    gg = [torch.cat([g[i] for g in grids_g], dim=1).contiguous() for i in range(3)]
    dt = periodic.median_spacing(t0s)
    ora = periodic.periodic_search(t0s, go["depth"], go["var"], go["dlnl"], periods, dt)
    res = api.nu_periodic_search(cu(t0s), Ds, *gg, cu(periods), phase_step=dt)
    gpu = {k: t.cpu().numpy() for k, t in res.items()}
    wl, wq, differ = periodic_compare(gpu, ora, t0s, go["depth"], go["var"], go["dlnl"],
                                      periods, dt, FP64_TOL, FP64_TOL, periodic.fold_period)
    best = periodic.best(ora, periods)
    print(f"per-sector factors, one fold: lnP err {wl:.2e}, Q err {wq:.2e}, ties {differ}, "
          f"best {best['period']:.4f}")
    assert abs(best["period"] - P) < 0.01


@pytest.mark.parametrize("symmetric", [False, True])
def test_rotation_alias_filter_is_bit_exact(symmetric):
    rng = np.random.default_rng(17)
    P_star = 1.37
    P = np.concatenate([rng.uniform(0.2, 13.5, 20000),
                        P_star * np.arange(1, 10),                 # exact multiples
                        P_star * np.arange(1, 10) * (1 - 0.02),    # at the edge
                        P_star * np.arange(1, 10) * (1 + 0.0199),
                        [np.nan, np.inf, -1.0]])
    got = api.nu_rotation_alias_filter(cu(P), P_star, 0.02, symmetric=symmetric).cpu().numpy()
    want = P[periodic.rotation_alias_keep(P, P_star, 0.02, symmetric)]
    assert got.shape == want.shape
    assert np.array_equal(got, want, equal_nan=True)
    assert 0 < len(want) < len(P)


def test_rotation_alias_filter_edge_cases():
    # everything dropped, a single period, bad arguments
    P = cu(2.0 * np.arange(1, 50))
    assert api.nu_rotation_alias_filter(P, 2.0).numel() == 0
    assert api.nu_rotation_alias_filter(cu([0.7]), 2.0).cpu().numpy().tolist() == [0.7]
    with pytest.raises(api.NuanceError):
        api.nu_rotation_alias_filter(P, 0.0)
    with pytest.raises(api.NuanceError):
        api.nu_rotation_alias_filter(P, 2.0, tol=float("nan"))
