"""Seven-sector light curve (N = 136 080, 20 durations): the dense oracle
does not fit (148 GB), so the linear search is checked on sampled templates
against the sequential celerite reference (oracle/semisep.py, itself pinned
to the dense oracle on smaller curves), and the fold on sampled periods of a
seeded grid of the same shape.  Parity here is pinned only indirectly."""
import numpy as np
import pytest

from oracle import periodic, semisep
from paper_2402_06835_gb300 import synth
from parity import FP64_TOL, linear_errors, periodic_compare

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def cu(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def test_multisector_linear_search_fp64_sampled():
    w = synth.multisector_136080()
    lc = w.curves[0]
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    d, v, l = api.nu_linear_search(f, cu(lc.t), w.durations)
    info = f.info()
    assert info["status"] == 0
    rng = np.random.default_rng(7)
    n = len(lc.t)
    edges = [0, n - 1, 19439, 19440, 20159, 20160, 68039, 136079 - 9720]
    idx = np.concatenate([rng.integers(0, n, 40), edges])
    pairs = [(int(rng.integers(0, len(w.durations))), int(i)) for i in idx]
    od, ov, ol, model = semisep.sampled_linear_search(lc.t, lc.y, lc.diag_var, lc.terms,
                                                      lc.X, w.durations, pairs)
    g = [a.cpu().numpy() for a in (d, v, l)]
    gsel = [np.array([a[j, i] for (j, i) in pairs]) for a in g]
    err = linear_errors(gsel, (od, ov, ol))
    print("multisector fp64 sampled errors", err)
    assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
    assert info["logdet"] == pytest.approx(model.logdet, rel=1e-11)
    assert info["lnL_null"] == pytest.approx(model.lnL_null, rel=1e-11)


def test_multisector_fold_fp64_sampled_periods():
    w = synth.multisector_136080()
    t0s = w.curves[0].t
    n = len(t0s)
    rng = np.random.default_rng(11)
    nD = len(w.durations)
    g = dict(depth=rng.normal(0, 5e-4, (nD, n)), var=rng.uniform(2e-8, 9e-8, (nD, n)),
             dlnl=rng.uniform(0, 6, (nD, n)))
    sel = np.concatenate([[0, len(w.periods) - 1], rng.integers(0, len(w.periods), 6)])
    periods = w.periods[sel]
    dt = periodic.median_spacing(t0s)
    res = api.nu_periodic_search(cu(t0s), w.durations, cu(g["depth"]), cu(g["var"]),
                                 cu(g["dlnl"]), cu(periods), phase_step=dt)
    gpu = {k: v.cpu().numpy() for k, v in res.items()}
    ora = periodic.periodic_search(t0s, g["depth"], g["var"], g["dlnl"], periods, dt)
    wl, wq, dif = periodic_compare(gpu, ora, t0s, g["depth"], g["var"], g["dlnl"], periods, dt,
                                   FP64_TOL, FP64_TOL, periodic.fold_period)
    print(f"multisector fold fp64: lnP err {wl:.2e} Q err {wq:.2e} ties {dif}")
