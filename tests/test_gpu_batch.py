"""GPU tests of the batched survey search (nu_batch_search).

The batch runs the same kernel bodies as the single-curve calls on packed
curves, so in FP64 its results must equal those of one nu_gp_factor +
nu_linear_search + nu_periodic_search per curve; two curves are also checked
against the oracle (FP64 1e-9, mixed 1e-3 absolute on Q), and a curve whose
times are unsorted must fail alone.
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

DS = np.array([0.02, 0.045, 0.07])
PERIODS = np.linspace(0.11, 0.9, 157)


def _curves():
    out = []
    for c, (n, gap, p_rot, sig) in enumerate([(300, None, 0.4, 1e-2), (520, 40, 0.9, 2e-2),
                                               (410, 25, 0.2, 5e-3), (677, 90, 1.7, 3e-2),
                                               (333, None, 0.6, 8e-3)]):
        out.append(synth.small_curve(n=n, seed=100 + c, p_rot=p_rot, sigma=sig, gap=gap,
                                     inject=(2.5e-3, 1.0 / 24.0, 0.37)))
    return out


def _single(lc, precision, dt):
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    d, v, l = api.nu_linear_search(f, cu(lc.t), DS, precision=precision)
    r = api.nu_periodic_search(cu(lc.t), DS, d, v, l, cu(PERIODS), precision=precision,
                               phase_step=dt)
    return {k: x.cpu().numpy() for k, x in r.items()}


@pytest.fixture(scope="module")
def curves():
    return _curves()


def test_batch_fp64_equals_single_curve_calls(curves):
    dt = synth.CADENCE_DAYS
    res = api.nu_batch_search([(lc.t, lc.y, lc.diag_var, lc.terms) for lc in curves], DS,
                              PERIODS, k=2, precision="fp64", phase_step=dt)
    assert res["status"] == [0] * len(curves)
    for c, lc in enumerate(curves):
        one = _single(lc, "fp64", dt)
        assert np.array_equal(res["D_idx"][c].cpu().numpy(), one["D_idx"])
        for key in ("Q", "T0", "lnP", "depth", "sigma"):
            a, b = res[key][c].cpu().numpy(), one[key]
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0, err_msg=key)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_against_oracle(curves, precision):
    dt = synth.CADENCE_DAYS
    res = api.nu_batch_search([(lc.t, lc.y, lc.diag_var, lc.terms) for lc in curves], DS,
                              PERIODS, k=2, precision=precision, phase_step=dt)
    for c in (1, 3):
        lc = curves[c]
        g = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, DS)
        ora = periodic.periodic_search(lc.t, g["depth"], g["var"], g["dlnl"], PERIODS, dt)
        gpu = {k: res[k][c].cpu().numpy() for k in ("Q", "T0", "D_idx", "depth", "sigma", "lnP")}
        if precision == "fp64":
            wl, wq, dif = periodic_compare(gpu, ora, lc.t, g["depth"], g["var"], g["dlnl"],
                                           PERIODS, dt, FP64_TOL, FP64_TOL, periodic.fold_period)
        else:
            wl, wq, dif = periodic_compare(gpu, ora, lc.t, g["depth"], g["var"], g["dlnl"],
                                           PERIODS, dt, 1e-4, MIXED_SNR_ABS,
                                           periodic.fold_period, max_reeval=len(PERIODS),
                                           q_abs=True)
        print(f"batch {precision} curve {c}: lnP err {wl:.2e} Q err {wq:.2e} ties {dif}")


def test_batch_reports_a_failing_curve_alone(curves):
    dt = synth.CADENCE_DAYS
    bad = curves[2]
    t = bad.t.copy()
    t[100], t[101] = t[101], t[100]
    items = [(lc.t, lc.y, lc.diag_var, lc.terms) for lc in curves]
    items[2] = (t, bad.y, bad.diag_var, bad.terms)
    res = api.nu_batch_search(items, DS, PERIODS, k=2, precision="fp64", phase_step=dt)
    st = res["status"]
    assert st[2] != 0 and all(s == 0 for i, s in enumerate(st) if i != 2)


def test_injection_workload_shape_against_oracle():
    """The injection-recovery set-up (4-day curves, SHO kernels with Q up to
    100 and amplitudes up to 12 % of the flux, one duration) through the batch:
    every curve equals its single-curve calls, two equal the oracle."""
    w = synth.injection_4000(n_curves=6)
    Ds = w.durations
    periods = np.linspace(0.3, 3.0, 300)
    dt = synth.CADENCE_DAYS
    res = api.nu_batch_search([(lc.t, lc.y, lc.diag_var, lc.terms) for lc in w.curves], Ds,
                              periods, k=2, precision="fp64", phase_step=dt)
    assert res["status"] == [0] * len(w.curves)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    for c, lc in enumerate(w.curves):
        f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
        d, v, l = api.nu_linear_search(f, cu(lc.t), Ds)
        one = api.nu_periodic_search(cu(lc.t), Ds, d, v, l, cu(periods), phase_step=dt)
        for key in ("Q", "T0", "lnP"):
            np.testing.assert_allclose(res[key][c].cpu().numpy(), one[key].cpu().numpy(),
                                       rtol=1e-12, atol=0, err_msg=key)
    for c in (0, 3):
        lc = w.curves[c]
        g = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds)
        ora = periodic.periodic_search(lc.t, g["depth"], g["var"], g["dlnl"], periods, dt)
        gpu = {k: res[k][c].cpu().numpy() for k in ("Q", "T0", "D_idx", "depth", "sigma", "lnP")}
        wl, wq, _ = periodic_compare(gpu, ora, lc.t, g["depth"], g["var"], g["dlnl"], periods,
                                     dt, FP64_TOL, FP64_TOL, periodic.fold_period)
        print(f"injection curve {c} (tau {lc.injected['tau']:.2f}, delta "
              f"{lc.injected['delta']:.2f}, Q {lc.injected['Q']:.1f}): lnP err {wl:.2e}, "
              f"Q err {wq:.2e}")
        assert wl <= FP64_TOL and wq <= FP64_TOL


def test_batch_with_wide_tree_levels():
    """75 000 samples in one batch: the factor scans' widest tree level has
    more than 4096 groups (one thread per group) and the upper levels fewer
    (one warp per group); every curve equals its single-curve calls, whose
    trees are warp-level throughout."""
    curves = [synth.small_curve(n=2500, seed=300 + c, p_rot=0.3 + 0.05 * c, sigma=8e-3,
                                gap=(60 if c % 3 == 0 else None),
                                inject=(2.5e-3, 1.0 / 24.0, 0.37))
              for c in range(30)]
    dt = synth.CADENCE_DAYS
    res = api.nu_batch_search([(lc.t, lc.y, lc.diag_var, lc.terms) for lc in curves], DS,
                              PERIODS, k=2, precision="fp64", phase_step=dt)
    assert res["status"] == [0] * len(curves)
    for c in (0, 7, 29):
        one = _single(curves[c], "fp64", dt)
        assert np.array_equal(res["D_idx"][c].cpu().numpy(), one["D_idx"])
        for key in ("Q", "T0", "lnP", "depth", "sigma"):
            np.testing.assert_allclose(res[key][c].cpu().numpy(), one[key], rtol=1e-12, atol=0,
                                       err_msg=key)


def test_batch_default_phase_step_is_first_curve_median(curves):
    """phase_step = 0 (None in the binding): the library takes the median
    sample spacing of the first curve, as the explicit value does."""
    items = [(lc.t, lc.y, lc.diag_var, lc.terms) for lc in curves]
    dt = float(np.median(np.diff(curves[0].t)))
    a = api.nu_batch_search(items, DS, PERIODS, k=2, precision="fp64", phase_step=None)
    b = api.nu_batch_search(items, DS, PERIODS, k=2, precision="fp64", phase_step=dt)
    for key in ("Q", "T0", "D_idx", "lnP", "depth", "sigma"):
        assert torch.equal(a[key], b[key]), key


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_graph_reuse_across_calls(precision):
    """The executable graph of a configuration is kept and updated with each
    call's buffers: two batches of the same shape and different data, called
    alternately (and with fresh output tensors every time), each give the
    results of their own first call, and in FP64 those of the single-curve
    calls."""
    dt = synth.CADENCE_DAYS
    sets = []
    for base in (200, 260):
        cs = [synth.small_curve(n=n, seed=base + c, p_rot=0.3 + 0.1 * c, sigma=6e-3,
                                gap=(30 if c == 1 else None), inject=(3e-3, 1.0 / 24.0, 0.41))
              for c, n in enumerate((350, 420, 380))]
        sets.append(cs)
    runs = []
    for rep in range(2):
        for cs in sets:
            r = api.nu_batch_search([(lc.t, lc.y, lc.diag_var, lc.terms) for lc in cs], DS,
                                    PERIODS, k=2, precision=precision, phase_step=dt)
            runs.append({k: v.cpu().numpy() for k, v in r.items() if k != "status"})
    for i in (0, 1):
        for key in ("Q", "T0", "D_idx", "lnP", "depth", "sigma"):
            assert np.array_equal(runs[i][key], runs[i + 2][key], equal_nan=True), key
    assert not np.array_equal(runs[0]["Q"], runs[1]["Q"])
    if precision == "fp64":
        for i, cs in enumerate(sets):
            for c, lc in enumerate(cs):
                one = _single(lc, "fp64", dt)
                np.testing.assert_allclose(runs[i]["Q"][c], one["Q"], rtol=1e-12, atol=0)


def test_injection_workload_mixed_against_oracle():
    """Mixed precision on the injection set-up (deep transits: many cells of
    every warp survive the first pass in the same round, which exercises the
    fold's queue flushing): every curve succeeds, two equal the FP64 oracle
    within the mixed tolerances."""
    w = synth.injection_4000(n_curves=48)
    Ds = w.durations
    periods = np.linspace(0.3, 3.0, 600)
    dt = synth.CADENCE_DAYS
    res = api.nu_batch_search([(lc.t, lc.y, lc.diag_var, lc.terms) for lc in w.curves], Ds,
                              periods, k=2, precision="mixed", phase_step=dt)
    assert res["status"] == [0] * len(w.curves)
    assert torch.isfinite(res["Q"]).all()
    for c in (5, 31):
        lc = w.curves[c]
        g = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds)
        ora = periodic.periodic_search(lc.t, g["depth"], g["var"], g["dlnl"], periods, dt)
        gpu = {k: res[k][c].cpu().numpy() for k in ("Q", "T0", "D_idx", "depth", "sigma", "lnP")}
        periodic_compare(gpu, ora, lc.t, g["depth"], g["var"], g["dlnl"], periods, dt, 1e-4,
                         MIXED_SNR_ABS, periodic.fold_period, max_reeval=len(periods),
                         q_abs=True)
        print(f"injection mixed curve {c}:", periodic_compare.last)
