"""Seven-sector light curve (N = 136 080, 20 durations): the dense oracle
does not fit (148 GB), so the linear search is checked on sampled templates
against the sequential celerite reference (oracle/semisep.py, itself pinned
to the dense oracle on smaller curves), in FP64 and in mixed precision, and
the fold on sampled periods of seeded grids of the same shape: one random,
one with periodic dips whose gains follow their depths (strong pruning, as on
a real light curve).  Parity here is pinned only indirectly."""
import numpy as np
import pytest

from oracle import periodic, semisep
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


@pytest.fixture(scope="module")
def ms():
    """The workload, sampled (duration, epoch) pairs and the celerite
    reference's values for them."""
    w = synth.multisector_136080()
    lc = w.curves[0]
    rng = np.random.default_rng(7)
    n = len(lc.t)
    edges = [0, n - 1, 19439, 19440, 20159, 20160, 68039, 136079 - 9720]
    idx = np.concatenate([rng.integers(0, n, 40), edges])
    pairs = [(int(rng.integers(0, len(w.durations))), int(i)) for i in idx]
    # the longest duration (windows of 120 samples) at every edge
    pairs += [(len(w.durations) - 1, int(i)) for i in edges]
    od, ov, ol, model = semisep.sampled_linear_search(lc.t, lc.y, lc.diag_var, lc.terms,
                                                      lc.X, w.durations, pairs)
    return w, lc, pairs, (od, ov, ol), model


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multisector_linear_search_sampled(ms, precision):
    w, lc, pairs, ora, model = ms
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    d, v, l = api.nu_linear_search(f, cu(lc.t), w.durations, precision=precision)
    info = f.info()
    assert info["status"] == 0
    g = [a.double().cpu().numpy() for a in (d, v, l)]
    gsel = [np.array([a[j, i] for (j, i) in pairs]) for a in g]
    err = linear_errors(gsel, ora)
    print(f"multisector {precision} sampled errors", err)
    if precision == "fp64":
        assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
        assert info["logdet"] == pytest.approx(model.logdet, rel=1e-11)
        assert info["lnL_null"] == pytest.approx(model.lnL_null, rel=1e-11)
    else:
        assert err["depth"] <= MIXED_DEPTH_TOL, err
        assert err["var"] <= 1e-4 and err["dlnl"] <= 1e-3, err


def _grid(kind, w, t0s, rng):
    nD, n = len(w.durations), len(t0s)
    if kind == "random":
        return dict(depth=rng.normal(0, 5e-4, (nD, n)), var=rng.uniform(2e-8, 9e-8, (nD, n)),
                    dlnl=rng.uniform(0, 6, (nD, n)))
    # noise depths with gains that follow them, plus a periodic dip (3.1 d)
    var = rng.uniform(2e-8, 9e-8, (nD, n))
    depth = rng.normal(0, 1, (nD, n)) * np.sqrt(var)
    ph = np.mod(t0s - 1.3, 3.1)
    dip = (ph < 0.05) | (ph > 3.1 - 0.05)
    depth[:, dip] += 1.2e-3
    depth[3, 5000:5040] = np.nan
    return dict(depth=depth, var=var, dlnl=depth ** 2 / (2 * var))


@pytest.mark.parametrize("kind", ["random", "dips"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multisector_fold_sampled_periods(kind, precision):
    w = synth.multisector_136080()
    t0s = w.curves[0].t
    rng = np.random.default_rng(11 if kind == "random" else 12)
    g = _grid(kind, w, t0s, rng)
    near = np.argmin(np.abs(w.periods - 3.1))
    sel = np.unique(np.concatenate([[0, len(w.periods) - 1, near - 1, near, near + 1],
                                    rng.integers(0, len(w.periods), 35)]))
    periods = w.periods[sel]
    dt = periodic.median_spacing(t0s)
    if precision == "mixed":
        g = {k: a.astype(np.float32).astype(np.float64) for k, a in g.items()}
    dty = torch.float64 if precision == "fp64" else torch.float32
    res = api.nu_periodic_search(cu(t0s), w.durations, cu(g["depth"], dty), cu(g["var"], dty),
                                 cu(g["dlnl"], dty), cu(periods), precision=precision,
                                 phase_step=dt)
    gpu = {k: v.cpu().numpy() for k, v in res.items()}
    ora = periodic.periodic_search(t0s, g["depth"], g["var"], g["dlnl"], periods, dt)
    if precision == "fp64":
        wl, wq, dif = periodic_compare(gpu, ora, t0s, g["depth"], g["var"], g["dlnl"], periods,
                                       dt, FP64_TOL, FP64_TOL, periodic.fold_period)
    else:
        wl, wq, dif = periodic_compare(gpu, ora, t0s, g["depth"], g["var"], g["dlnl"], periods,
                                       dt, 1e-4, MIXED_SNR_ABS, periodic.fold_period,
                                       max_reeval=len(periods), q_abs=True,
                                       tol_ds=MIXED_DEPTH_TOL)
    print(f"multisector fold {precision} {kind}:", periodic_compare.last)
