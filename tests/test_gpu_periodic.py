"""GPU parity of the periodic search (Sect. 2.3-2.4) against the oracle fold.

The fold's inputs are single-event grids computed by the oracle (or drawn at
random by the seeded generator for full-size shapes); both sides fold the
same grid.  ln P of the best cell is unique and is compared directly; when
the GPU's argmax cell differs from the oracle's (a near-tie), the oracle is
evaluated at the GPU's cell and must give the same maximum and Q.
"""
import numpy as np
import pytest

from oracle import linear, periodic
from paper_2402_06835_gb300 import synth
from parity import FP64_TOL, MIXED_SNR_ABS, periodic_compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def cu(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.fixture(scope="module")
def c1_grid():
    w = synth.single_2048()
    lc = w.curves[0]
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t,
                               w.durations)
    return w, lc, ora


def _gpu_fold(t0s, Ds, grid, periods, precision, phase_step=0.0):
    dt = torch.float64 if precision == "fp64" else torch.float32
    res = api.nu_periodic_search(cu(t0s), Ds, cu(grid["depth"], dt), cu(grid["var"], dt),
                                 cu(grid["dlnl"], dt), cu(periods), precision=precision,
                                 phase_step=phase_step)
    return {k: v.cpu().numpy() for k, v in res.items()}


def test_fold_fp64_single_2048(c1_grid):
    w, lc, g = c1_grid
    dt = periodic.median_spacing(lc.t)
    ora = periodic.periodic_search(lc.t, g["depth"], g["var"], g["dlnl"], w.periods, dt)
    gpu = _gpu_fold(lc.t, w.durations, g, w.periods, "fp64")
    wl, wq, differ = periodic_compare(gpu, ora, lc.t, g["depth"], g["var"], g["dlnl"],
                                      w.periods, dt, FP64_TOL, FP64_TOL,
                                      periodic.fold_period)
    print(f"single_2048 fold fp64: lnP err {wl:.2e}, Q err {wq:.2e}, argmax ties {differ}")
    b_o = periodic.best(ora, w.periods)
    b_g = int(np.argmax(np.where(np.isfinite(gpu["Q"]), gpu["Q"], -np.inf)))
    assert abs(w.periods[b_g] - b_o["period"]) < 1e-12 or differ > 0


def test_fold_mixed_single_2048(c1_grid):
    w, lc, g = c1_grid
    dt = periodic.median_spacing(lc.t)
    ora = periodic.periodic_search(lc.t, g["depth"], g["var"], g["dlnl"], w.periods, dt)
    gpu = _gpu_fold(lc.t, w.durations, g, w.periods, "mixed")
    wl, wq, differ = periodic_compare(gpu, ora, lc.t, g["depth"], g["var"], g["dlnl"],
                                      w.periods, dt, 1e-4, MIXED_SNR_ABS,
                                      periodic.fold_period, max_reeval=1000, q_abs=True)
    print(f"single_2048 fold mixed: lnP err {wl:.2e}, Q abs err {wq:.2e}, ties {differ}")


def test_end_to_end_single_2048_recovers_injection(c1_grid):
    w, lc, g = c1_grid
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    d, v, l = api.nu_linear_search(f, cu(lc.t), w.durations)
    res = api.nu_periodic_search(cu(lc.t), w.durations, d, v, l, cu(w.periods))
    Q = res["Q"].cpu().numpy()
    p = int(np.argmax(Q))
    inj = lc.injected["period"]
    # best period at the injected one or a simple alias
    ratios = np.array([1.0, 0.5, 2.0])
    assert np.min(np.abs(w.periods[p] / inj - ratios)) < 0.02, (w.periods[p], inj)


def test_fold_gaps_edges_and_explicit_step():
    """Random grid with a gap and NaN holes; explicit phase step."""
    rng = np.random.default_rng(17)
    t0s = np.concatenate([np.arange(700), np.arange(900, 1500)]) * synth.CADENCE_DAYS
    n = len(t0s)
    g = dict(depth=rng.normal(0, 1e-3, (3, n)), var=rng.uniform(1e-8, 5e-8, (3, n)),
             dlnl=rng.uniform(0, 8, (3, n)))
    g["depth"][1, 100:110] = np.nan
    g["var"][2, 650:720] = np.nan
    periods = np.linspace(0.05, 1.9, 257)
    dt = synth.CADENCE_DAYS
    ora = periodic.periodic_search(t0s, g["depth"], g["var"], g["dlnl"], periods, dt)
    gpu = _gpu_fold(t0s, np.ones(3), g, periods, "fp64", phase_step=dt)
    periodic_compare(gpu, ora, t0s, g["depth"], g["var"], g["dlnl"], periods, dt,
                     FP64_TOL, FP64_TOL, periodic.fold_period)


def test_fold_no_valid_cell():
    t0s = np.arange(50) * synth.CADENCE_DAYS
    nan = np.full((1, 50), np.nan)
    g = dict(depth=nan, var=nan, dlnl=nan)
    gpu = _gpu_fold(t0s, np.ones(1), g, np.array([0.02, 0.03]), "fp64")
    assert np.all(gpu["Q"] == 0.0) and np.all(gpu["D_idx"] == -1)
    assert np.all(np.isneginf(gpu["lnP"]))


@pytest.mark.slow
def test_fold_fp64_sector_shape_sampled_periods():
    """Full sector shape (19 440 epochs with a 1-day gap, 10 durations, 20 000
    periods) on a seeded random grid; the oracle checks 40 sampled periods."""
    w = synth.sector_19440()
    t0s = w.curves[0].t
    n = len(t0s)
    rng = np.random.default_rng(5)
    g = dict(depth=rng.normal(0, 5e-4, (10, n)), var=rng.uniform(2e-8, 9e-8, (10, n)),
             dlnl=rng.uniform(0, 6, (10, n)))
    gpu = _gpu_fold(t0s, w.durations, g, w.periods, "fp64")
    dt = periodic.median_spacing(t0s)
    sel = np.concatenate([[0, 1, len(w.periods) - 1], rng.integers(0, len(w.periods), 37)])
    ora = periodic.periodic_search(t0s, g["depth"], g["var"], g["dlnl"], w.periods[sel], dt)
    gsel = {k: v[sel] for k, v in gpu.items()}
    wl, wq, differ = periodic_compare(gsel, ora, t0s, g["depth"], g["var"], g["dlnl"],
                                      w.periods[sel], dt, FP64_TOL, FP64_TOL,
                                      periodic.fold_period)
    print(f"sector fold fp64 sampled: lnP err {wl:.2e}, Q err {wq:.2e}, ties {differ}")


@pytest.mark.parametrize("jitter", [0.0, 0.3])
def test_fold_mixed_gapped_and_irregular(jitter):
    """Mixed precision on a gapped grid with NaN holes: the fixed-point slot
    walk (regular epochs) and the exact FP64-epoch walk (jittered epochs)."""
    rng = np.random.default_rng(23)
    dt = synth.CADENCE_DAYS
    t0s = np.concatenate([np.arange(900), np.arange(1100, 1900)]) * dt
    t0s = t0s + jitter * dt * rng.uniform(-1, 1, len(t0s)) * (np.arange(len(t0s)) % 3 == 1)
    n = len(t0s)
    g = dict(depth=rng.normal(0, 1e-3, (4, n)), var=rng.uniform(1e-8, 5e-8, (4, n)),
             dlnl=rng.uniform(0, 8, (4, n)))
    g["depth"][2, 300:320] = np.nan
    periods = np.concatenate([np.linspace(0.03, 1.0, 200), [2.3, 2.61, 3.9]])
    ora = periodic.periodic_search(t0s, g["depth"], g["var"], g["dlnl"], periods, dt)
    gpu = _gpu_fold(t0s, np.ones(4), g, periods, "mixed", phase_step=dt)
    wl, wq, differ = periodic_compare(gpu, ora, t0s, g["depth"], g["var"], g["dlnl"],
                                      periods, dt, 1e-4, MIXED_SNR_ABS, periodic.fold_period,
                                      max_reeval=len(periods), q_abs=True)
    print(f"mixed fold jitter={jitter}: lnP err {wl:.2e}, Q abs err {wq:.2e}, ties {differ}")


def test_fold_invalid_periods_are_nan():
    t0s = np.arange(200) * synth.CADENCE_DAYS
    rng = np.random.default_rng(2)
    g = dict(depth=rng.normal(0, 1e-3, (1, 200)), var=np.full((1, 200), 1e-8),
             dlnl=rng.uniform(0, 2, (1, 200)))
    periods = np.array([0.05, -1.0, np.nan, 1e-300, 0.07])
    for prec in ("fp64", "mixed"):
        gpu = _gpu_fold(t0s, np.ones(1), g, periods, prec, phase_step=synth.CADENCE_DAYS)
        assert np.isnan(gpu["Q"][1:4]).all() and (gpu["D_idx"][1:4] == -1).all()
        assert np.isfinite(gpu["Q"][[0, 4]]).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fold_period_order_does_not_change_results(precision):
    """The folds take a descending period grid from its far end (short periods
    first); every period's outputs are the same in any order of the grid:
    ascending, descending, shuffled, and with NaN entries at either end."""
    rng = np.random.default_rng(5)
    dt = synth.CADENCE_DAYS
    t0s = np.concatenate([np.arange(900), np.arange(960, 1700)]) * dt
    n = len(t0s)
    var = rng.uniform(1e-8, 5e-8, (3, n))
    depth = rng.normal(0, 1.5e-4, (3, n))
    depth[:, 400:406] += 1.5e-3
    g = dict(depth=depth, var=var, dlnl=depth ** 2 / (2 * var))
    if precision == "mixed":
        g = {k: a.astype(np.float32).astype(np.float64) for k, a in g.items()}
    P = np.linspace(0.04, 1.5, 700)
    ref = _gpu_fold(t0s, np.ones(3), g, P, precision, phase_step=dt)
    perm = rng.permutation(len(P))
    for order in (np.arange(len(P))[::-1], perm):
        out = _gpu_fold(t0s, np.ones(3), g, P[order], precision, phase_step=dt)
        for k in ref:
            np.testing.assert_array_equal(out[k], ref[k][order], err_msg=k)
    Pn = np.concatenate([[np.nan], P[::-1], [np.nan]])
    out = _gpu_fold(t0s, np.ones(3), g, Pn, precision, phase_step=dt)
    assert np.isnan(out["Q"][[0, -1]]).all()
    for k in ref:
        np.testing.assert_array_equal(out[k][1:-1], ref[k][::-1], err_msg=k)


@pytest.mark.parametrize("drift", [0.0, 3e-10])
@pytest.mark.parametrize("offset", [0.0, 2000.0])
@pytest.mark.parametrize("regular", [True, False])
def test_fold_fp64_screen_hard_cases(offset, regular, drift):
    """FP64 fold on grids built to stress the FP32 screen of the exact path:
    periods that are whole multiples of the step (epochs land on samples and
    on the edges of gaps and NaN holes), epochs far from zero, regular
    epochs (slot-indexed screen) or irregular ones with near-coincident pairs
    (position search), neighbours whose variances differ by orders of
    magnitude, and gains consistent with the depths (strong pruning) next to
    unrelated ones.  With drift the phase step differs from the cadence by
    that fraction, so the samples sit up to 5e-7 step off the phase grid (as
    a median spacing of FP64 times puts them on long curves).  Every period
    is compared."""
    rng = np.random.default_rng(41)
    dt = synth.CADENCE_DAYS
    base = np.concatenate([np.arange(600), np.arange(640, 1300), np.arange(1302, 1500)])
    t0s = offset + base * dt
    if not regular:
        t0s[5::97] += 0.9 * dt      # near-coincident pairs (gap 0.1 dt)
        t0s = np.sort(t0s)
    n = len(t0s)
    var = rng.uniform(1e-8, 5e-8, (4, n))
    var[1, ::53] *= 1e4             # isolated very noisy samples
    depth = rng.normal(0, 1e-4, (4, n))
    depth[:, 300:310] += 2e-3       # one strong event
    dlnl = depth ** 2 / (2 * var)
    dlnl[3] = rng.uniform(0, 8, n)  # unrelated gains in the last row
    depth[2, 100:110] = np.nan
    var[0, 598:603] = np.nan        # hole next to the first gap
    g = dict(depth=depth, var=var, dlnl=dlnl)
    periods = np.concatenate([np.arange(37, 400, 3) * dt,
                              np.linspace(0.05, 1.2, 150), [1.9, 2.05]])
    step = dt * (1.0 + drift)
    ora = periodic.periodic_search(t0s, depth, var, dlnl, periods, step)
    gpu = _gpu_fold(t0s, np.ones(4), g, periods, "fp64", phase_step=step)
    wl, wq, differ = periodic_compare(gpu, ora, t0s, depth, var, dlnl, periods, step,
                                      FP64_TOL, FP64_TOL, periodic.fold_period)
    print(f"fp64 screen hard cases offset={offset} regular={regular} drift={drift}: "
          f"lnP err {wl:.2e}, Q err {wq:.2e}, ties {differ}")


def test_fold_fp64_peak_seed_edges():
    """One event dominates every cell that catches it (the case the FP64
    fold's peak seed is for), placed at the last epoch of the last duration
    row; an equal gain earlier in the grid (the seed takes the first), and
    infinite gains (never a seed, dropped by both sides).  Periods short and
    long against the span, so that the seeded periods (cells of fewer than 32
    epochs) and the others are both compared."""
    rng = np.random.default_rng(43)
    dt = synth.CADENCE_DAYS
    t0s = 3.0 + np.arange(1200) * dt
    n = len(t0s)
    var = rng.uniform(1e-8, 5e-8, (3, n))
    depth = rng.normal(0, 1e-4, (3, n))
    depth[2, -1] = 3e-3
    depth[0, 500], var[0, 500] = depth[2, -1], var[2, -1]
    dlnl = depth ** 2 / (2 * var)
    dlnl[1, 10] = np.inf
    dlnl[0, 900] = -np.inf
    g = dict(depth=depth, var=var, dlnl=dlnl)
    periods = np.concatenate([np.linspace(0.03, 0.06, 20), np.linspace(0.06, 1.6, 180)])
    ora = periodic.periodic_search(t0s, depth, var, dlnl, periods, dt)
    gpu = _gpu_fold(t0s, np.ones(3), g, periods, "fp64", phase_step=dt)
    wl, wq, differ = periodic_compare(gpu, ora, t0s, depth, var, dlnl, periods, dt,
                                      FP64_TOL, FP64_TOL, periodic.fold_period)
    print(f"fp64 peak seed edges: lnP err {wl:.2e}, Q err {wq:.2e}, ties {differ}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_period_grid_kernels(precision):
    """Grids of 8192 periods or more run the small-block fold instances (FP64:
    64 threads, 14 blocks per SM; mixed: 128 threads).  On 9000 periods they
    must give what the 256-thread instances give on the two halves of the grid,
    and the oracle's results at sampled periods."""
    lc = synth.small_curve(n=2200, seed=3, p_rot=1.3, sigma=4e-3, sigma_w=1e-3,
                           inject=(3e-3, 1.0 / 24.0, 0.41))
    Ds = np.array([0.03, 1.0 / 24.0, 0.055])
    periods = np.linspace(0.12, 3.0, 9000)
    dt = periodic.median_spacing(lc.t)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    d, v, l = api.nu_linear_search(f, cu(lc.t), Ds, precision=precision)
    whole = api.nu_periodic_search(cu(lc.t), Ds, d, v, l, cu(periods), precision=precision,
                                   phase_step=dt)
    halves = [api.nu_periodic_search(cu(lc.t), Ds, d, v, l, cu(periods[s]),
                                     precision=precision, phase_step=dt)
              for s in (slice(0, 4500), slice(4500, 9000))]
    for key in ("Q", "T0", "D_idx", "lnP", "depth", "sigma"):
        a = whole[key].cpu().numpy()
        b = np.concatenate([h[key].cpu().numpy() for h in halves])
        assert np.array_equal(a, b, equal_nan=True), key
    if precision == "fp64":
        sel = np.arange(0, 9000, 225)
        ora_lin = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds)
        ora = periodic.periodic_search(lc.t, ora_lin["depth"], ora_lin["var"], ora_lin["dlnl"],
                                       periods[sel], dt)
        gpu = {k: whole[k].cpu().numpy()[sel] for k in ("Q", "T0", "D_idx", "lnP", "depth",
                                                      "sigma")}
        wl, wq, _ = periodic_compare(gpu, ora, lc.t, ora_lin["depth"], ora_lin["var"],
                                     ora_lin["dlnl"], periods[sel], dt, FP64_TOL, FP64_TOL,
                                     periodic.fold_period)
        assert wl <= FP64_TOL and wq <= FP64_TOL
