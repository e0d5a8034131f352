"""Full-size parity of the sector workloads against the oracle's whole grid.

The dense oracle's whole-grid route (``oracle.linear.box_grid``: Sigma^-1 once,
then every box template of the grid) gives the linear search of a 19 440-sample
sector for every (t0, D), so the CUDA path is compared template by template,
and the fold (Sect. 2.3-2.4) runs on the linear-search output of a light curve
with an injected transit (strong pruning, as in real searches) instead of a
random grid:

* the FP64 sector (10 durations, 20 000 periods): every template of the FP64
  linear search; the FP64 fold on the oracle's grid; the whole FP64 chain
  (factor, linear search, fold on the GPU's own grid);
* the mixed-precision sector (16 durations, windows up to 90 samples): every
  template of the mixed linear search, the mixed fold on the oracle's grid
  rounded to FP32, and the whole mixed chain, each against the FP64 oracle
  with the mixed tolerances (1e-4 relative on depth, 1e-3 absolute on Q).

Periods are compared at a sample: 100 drawn at random, the neighbourhoods of
the injected period and its aliases, and the GPU's 20 best.  The worst errors
per output are printed (they are the per-output error figures of the mixed
path).
"""
import numpy as np
import pytest

from oracle import linear, periodic
from paper_2402_06835_gb300 import synth
from parity import (FP64_TOL, MIXED_DEPTH_TOL, MIXED_SNR_ABS, linear_errors,
                    periodic_compare)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def cu(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _oracle(w):
    lc = w.curves[0]
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    grid = linear.box_grid(model, lc.t, w.durations)
    return lc, model, grid


@pytest.fixture(scope="module")
def sector():
    w = synth.sector_19440()
    lc, model, grid = _oracle(w)
    return w, lc, model, grid


@pytest.fixture(scope="module")
def sector16():
    w = synth.sector_19440_16d()
    lc, model, grid = _oracle(w)
    return w, lc, model, grid


def _gpu_linear(lc, Ds, precision):
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    out = api.nu_linear_search(f, cu(lc.t), Ds, precision=precision)
    info = f.info()
    assert info["status"] == 0, info
    return out, info


def _periods_to_check(w, Q, seed):
    """Sampled period indices: random ones, the injected period's
    neighbourhood and its aliases', and the best 20 by the given Q."""
    rng = np.random.default_rng(seed)
    P = w.periods
    inj = w.curves[0].injected["period"]
    sel = list(rng.integers(0, len(P), 100))
    for target in (inj, inj / 2, 2 * inj):
        c = int(np.argmin(np.abs(P - target)))
        sel += list(range(max(0, c - 6), min(len(P), c + 7)))
    q = np.where(np.isfinite(Q), Q, -np.inf)
    sel += list(np.argsort(-q, kind="stable")[:20])
    sel += [0, len(P) - 1]
    return np.unique(np.array(sel, dtype=np.int64))


def _fold(t0s, Ds, grid, periods, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    res = api.nu_periodic_search(cu(t0s), Ds, cu(grid["depth"], dt), cu(grid["var"], dt),
                                 cu(grid["dlnl"], dt), cu(periods), precision=precision)
    return {k: v.cpu().numpy() for k, v in res.items()}


def _compare_fold(gpu, w, t0s, grid, sel, precision):
    dt = periodic.median_spacing(t0s)
    ora = periodic.periodic_search(t0s, grid["depth"], grid["var"], grid["dlnl"],
                                   w.periods[sel], dt)
    gsel = {k: v[sel] for k, v in gpu.items()}
    if precision == "fp64":
        periodic_compare(gsel, ora, t0s, grid["depth"], grid["var"], grid["dlnl"],
                         w.periods[sel], dt, FP64_TOL, FP64_TOL, periodic.fold_period)
    else:
        periodic_compare(gsel, ora, t0s, grid["depth"], grid["var"], grid["dlnl"],
                         w.periods[sel], dt, 1e-4, MIXED_SNR_ABS, periodic.fold_period,
                         max_reeval=len(sel), q_abs=True, tol_ds=MIXED_DEPTH_TOL)
    return dict(periodic_compare.last)


# ------------------------------------------------------------ FP64 sector
def test_sector_linear_fp64_every_template(sector):
    w, lc, model, grid = sector
    out, info = _gpu_linear(lc, w.durations, "fp64")
    err = linear_errors([o.cpu().numpy() for o in out],
                        (grid["depth"], grid["var"], grid["dlnl"]))
    print("sector_19440 fp64, every template:", err)
    assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
    assert info["logdet"] == pytest.approx(model.logdet, rel=1e-12)
    assert info["lnL_null"] == pytest.approx(model.lnL_null, rel=1e-12)


def test_sector_fold_fp64_on_oracle_grid(sector):
    w, lc, model, grid = sector
    gpu = _fold(lc.t, w.durations, grid, w.periods, "fp64")
    sel = _periods_to_check(w, gpu["Q"], 61)
    e = _compare_fold(gpu, w, lc.t, grid, sel, "fp64")
    print(f"sector_19440 fp64 fold on the oracle grid ({len(sel)} periods):", e)


def test_sector_chain_fp64(sector):
    """Factor, linear search and fold on the GPU against the oracle's linear
    search and fold; the injected planet (3.1 d) is the best period or an
    alias of it."""
    w, lc, model, grid = sector
    (d, v, l), _ = _gpu_linear(lc, w.durations, "fp64")
    res = api.nu_periodic_search(cu(lc.t), w.durations, d, v, l, cu(w.periods))
    gpu = {k: x.cpu().numpy() for k, x in res.items()}
    sel = _periods_to_check(w, gpu["Q"], 62)
    e = _compare_fold(gpu, w, lc.t, grid, sel, "fp64")
    print(f"sector_19440 fp64 chain ({len(sel)} periods):", e)
    best = w.periods[int(np.nanargmax(gpu["Q"]))]
    inj = lc.injected["period"]
    assert min(abs(best / inj - r) for r in (1.0, 0.5, 2.0)) < 0.01, best


# ----------------------------------------------------------- mixed sector
def test_sector16_linear_mixed_every_template(sector16):
    w, lc, model, grid = sector16
    out, _ = _gpu_linear(lc, w.durations, "mixed")
    err = linear_errors([o.double().cpu().numpy() for o in out],
                        (grid["depth"], grid["var"], grid["dlnl"]))
    print("sector_19440_16d mixed, every template:", err)
    assert err["depth"] <= MIXED_DEPTH_TOL, err
    assert err["var"] <= 1e-4 and err["dlnl"] <= 1e-3, err


def test_sector16_fold_mixed_on_oracle_grid(sector16):
    """The mixed fold's own error: both sides fold the oracle's grid rounded
    to FP32 (the oracle in FP64 on the rounded values)."""
    w, lc, model, grid = sector16
    g32 = {k: grid[k].astype(np.float32).astype(np.float64) for k in ("depth", "var", "dlnl")}
    gpu = _fold(lc.t, w.durations, g32, w.periods, "mixed")
    sel = _periods_to_check(w, gpu["Q"], 63)
    e = _compare_fold(gpu, w, lc.t, g32, sel, "mixed")
    print(f"sector_19440_16d mixed fold on the oracle grid ({len(sel)} periods):", e)


def test_sector16_chain_mixed(sector16):
    """The whole mixed chain against the FP64 oracle: the per-output error of
    the mixed path (depth, sigma, ln P of the fold; Q absolute)."""
    w, lc, model, grid = sector16
    (d, v, l), _ = _gpu_linear(lc, w.durations, "mixed")
    res = api.nu_periodic_search(cu(lc.t), w.durations, d, v, l, cu(w.periods),
                                 precision="mixed")
    gpu = {k: x.cpu().numpy() for k, x in res.items()}
    sel = _periods_to_check(w, gpu["Q"], 64)
    e = _compare_fold(gpu, w, lc.t, grid, sel, "mixed")
    print(f"sector_19440_16d mixed chain ({len(sel)} periods):", e)
