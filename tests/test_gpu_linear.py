"""GPU parity of the factor and the linear search against the dense oracle.

Every call goes through the C ABI (ctypes binding); every expected value comes
from ``oracle`` on the same seeded inputs.  FP64 mode must agree within 1e-9
(depth, variance, gain; norms in tests/parity.py), mixed mode within 1e-4 on
depth.
"""
import numpy as np
import pytest

from oracle import gp, linear
from paper_2402_06835_gb300 import synth
from parity import FP64_TOL, MIXED_DEPTH_TOL, linear_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def gpu_search(lc, t0s, Ds, terms=None, X=None, kind="box", ingress=0.1,
               precision="fp64"):
    terms = lc.terms if terms is None else terms
    X = lc.X if X is None else X
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), terms,
                         cu(X) if X.shape[1] else None, cu(lc.y))
    out = api.nu_linear_search(f, cu(t0s), Ds, template=kind, ingress_frac=ingress,
                               precision=precision)
    info = f.info()
    assert info["status"] == 0, info
    return [o.double().cpu().numpy() for o in out], info, f


CASES = {
    "rotation": dict(terms=None),
    "rotation+exp": dict(terms=[(gp.ROTATION, (1e-2, 0.5, 5.0, 0.0, 0.5)),
                                (gp.EXP, (2e-3, 0.08))]),
    "sho_overdamped": dict(terms=[(gp.SHO, (5e-3, 30.0, 0.3))]),
    "sho_critical": dict(terms=[(gp.SHO, (5e-3, 30.0, 0.5))]),
    "sho_q45": dict(terms=[(gp.SHO, (8e-3, 40.0, 45.0))]),
    "white_only": dict(terms=[]),
    # four 2x2 blocks: the largest state (J = 8)
    "two_rotations": dict(terms=[(gp.ROTATION, (1e-2, 0.5, 5.0, 0.0, 0.5)),
                                 (gp.ROTATION, (5e-3, 2.3, 3.0, 0.5, 0.3))]),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["box", "trapezoid", "limb_quad"])
def test_linear_fp64_small(case, kind):
    lc = synth.small_curve(n=300, seed=21, gap=40)
    terms = CASES[case]["terms"]
    terms = lc.terms if terms is None else terms
    Ds = np.array([0.01, 0.035, 0.07])
    # epochs: every sample, plus epochs in the gap and beyond both ends
    t0s = np.concatenate([lc.t, [0.5 * (lc.t[149] + lc.t[150]), lc.t[0] - 0.01,
                                 lc.t[-1] + 0.02]])
    gpu, info, _ = gpu_search(lc, t0s, Ds, terms=terms, kind=kind, ingress=0.2)
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, terms, lc.X, t0s, Ds,
                               kind=kind, ingress_frac=0.2)
    err = linear_errors(gpu, (ora["depth"], ora["var"], ora["dlnl"]))
    assert err["depth"] <= FP64_TOL and err["var"] <= FP64_TOL and err["dlnl"] <= FP64_TOL, err
    assert info["logdet"] == pytest.approx(ora["logdet"], rel=1e-11)
    assert info["lnL_null"] == pytest.approx(ora["lnL_null"], rel=1e-11)


def test_linear_no_design_matrix():
    lc = synth.small_curve(n=200, seed=4, design=False)
    Ds = np.array([0.02, 0.05])
    gpu, _, _ = gpu_search(lc, lc.t, Ds)
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds)
    err = linear_errors(gpu, (ora["depth"], ora["var"], ora["dlnl"]))
    assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err


def test_single_epoch_and_empty_window():
    lc = synth.small_curve(n=120, seed=6, gap=30)
    t0s = np.array([0.5 * (lc.t[59] + lc.t[60])])      # centre of the gap
    gpu, _, _ = gpu_search(lc, t0s, np.array([0.01]))
    assert np.isnan(gpu[0][0, 0]) and np.isnan(gpu[1][0, 0]) and np.isnan(gpu[2][0, 0])


@pytest.fixture(scope="module")
def c1():
    w = synth.single_2048()
    lc = w.curves[0]
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t,
                               w.durations)
    return w, lc, ora


def test_single_2048_fp64_full_grid(c1):
    w, lc, ora = c1
    gpu, info, _ = gpu_search(lc, lc.t, w.durations)
    err = linear_errors(gpu, (ora["depth"], ora["var"], ora["dlnl"]))
    print("single_2048 fp64 errors", err)
    assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
    assert info["logdet"] == pytest.approx(ora["logdet"], rel=1e-12)


def test_single_2048_mixed_full_grid(c1):
    w, lc, ora = c1
    gpu, _, _ = gpu_search(lc, lc.t, w.durations, precision="mixed")
    err = linear_errors(gpu, (ora["depth"], ora["var"], ora["dlnl"]))
    print("single_2048 mixed errors", err)
    assert err["depth"] <= MIXED_DEPTH_TOL, err
    assert err["var"] <= 1e-4 and err["dlnl"] <= 1e-3, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_limb_quad_coefficients(precision):
    """The limb-darkening coefficients reach the kernel: non-default (u1, u2)
    against the oracle, and u1 = u2 = 0 reproduces the box."""
    lc = synth.small_curve(n=500, seed=8, gap=25)
    Ds = np.array([0.02, 0.06])
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    g = [o.double().cpu().numpy() for o in
         api.nu_linear_search(f, cu(lc.t), Ds, template="limb_quad", ld=(0.62, -0.1),
                              precision=precision)]
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds,
                               kind="limb_quad", ld=(0.62, -0.1))
    err = linear_errors(g, (ora["depth"], ora["var"], ora["dlnl"]))
    if precision == "fp64":
        assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
    else:
        assert err["depth"] <= MIXED_DEPTH_TOL and err["var"] <= 1e-4, err
    flat = [o.double().cpu().numpy() for o in
            api.nu_linear_search(f, cu(lc.t), Ds, template="limb_quad", ld=(0.0, 0.0),
                                 precision=precision)]
    box = [o.double().cpu().numpy() for o in
           api.nu_linear_search(f, cu(lc.t), Ds, template="box", precision=precision)]
    for a, b in zip(flat, box):
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(b)
        assert np.allclose(a[ok], b[ok], rtol=1e-12 if precision == "fp64" else 1e-6, atol=0)
    with pytest.raises(api.NuanceError):
        api.nu_linear_search(f, cu(lc.t), Ds, template="limb_quad", ld=(float("nan"), 0.1))


def test_factor_rejects_unsorted_times():
    lc = synth.small_curve(n=64, seed=2)
    t = lc.t.copy()
    t[30], t[31] = t[31], t[30]
    f = api.nu_gp_factor(cu(t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    info = f.info()
    assert info["status"] == api.NU_EINVAL
    assert info["first_bad"] == 31


def test_factor_rejects_non_positive_definite():
    lc = synth.small_curve(n=64, seed=2)
    dv = lc.diag_var.copy()
    dv[40] = -1.0                    # negative variance: pivot <= 0 at 40
    f = api.nu_gp_factor(cu(lc.t), cu(dv), [], cu(lc.X), cu(lc.y))
    info = f.info()
    assert info["status"] == api.NU_ENOTPD
    assert info["first_bad"] == 40


@pytest.mark.slow
def test_sector_19440_fp64_sampled():
    """Full-size sector: GPU on the whole grid, oracle on sampled templates
    (dense Sigma of 19 440^2, one Cholesky)."""
    w = synth.sector_19440()
    lc = w.curves[0]
    gpu, info, _ = gpu_search(lc, lc.t, w.durations)
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    rng = np.random.default_rng(99)
    n = len(lc.t)
    idx = np.concatenate([rng.integers(0, n, 150), [0, 1, n - 1, n - 2, 9719, 9720]])
    pairs = [(int(rng.integers(0, len(w.durations))), int(i)) for i in idx]
    pairs += [(len(w.durations) - 1, 9719), (0, 9720), (len(w.durations) - 1, n - 1)]
    d, v, l = linear.sampled_linear_search(model, lc.t, w.durations, pairs)
    gsel = [np.array([g[j, i] for (j, i) in pairs]) for g in gpu]
    err = linear_errors(gsel, (d, v, l))
    print("sector_19440 fp64 sampled errors", err)
    assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
    assert info["logdet"] == pytest.approx(model.logdet, rel=1e-12)
    assert info["lnL_null"] == pytest.approx(model.lnL_null, rel=1e-12)


@pytest.mark.parametrize("case", ["rotation", "white_only", "sho_overdamped", "two_rotations",
                                  "rotation+exp"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_window_start_path(case, precision):
    """Epochs at the samples (the window-start recursion serves the box
    windows that are not clipped; the per-template kernel the others): a
    gapped curve with durations that give equal window lengths, one shorter
    than the cadence (no sample in most windows), several longer than one
    staged chunk (64 samples) and one close to the whole span."""
    lc = synth.small_curve(n=700, seed=29, gap=55)
    terms = CASES[case]["terms"]
    terms = lc.terms if terms is None else terms
    dt = synth.CADENCE_DAYS
    Ds = np.array([0.5 * dt, 7.2 * dt, 7.4 * dt, 7.3 * dt, 0.06, 70.5 * dt, 131 * dt,
                   0.45, 660 * dt])
    gpu, _, _ = gpu_search(lc, lc.t, Ds, terms=terms, precision=precision)
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, terms, lc.X, lc.t, Ds)
    err = linear_errors(gpu, (ora["depth"], ora["var"], ora["dlnl"]))
    print(f"window-start path {case} {precision}:", err)
    if precision == "fp64":
        assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
    else:
        assert err["depth"] <= MIXED_DEPTH_TOL and err["var"] <= 1e-4, err


@pytest.mark.parametrize("n", [5, 40, 64, 65, 200])
def test_linear_window_start_short_curves(n):
    """Curves shorter than, equal to and just above one block of window
    starts (64 on small curves)."""
    lc = synth.small_curve(n=n, seed=31)
    Ds = np.array([1.5 * synth.CADENCE_DAYS, 0.02, 0.05])
    gpu, _, _ = gpu_search(lc, lc.t, Ds)
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds)
    err = linear_errors(gpu, (ora["depth"], ora["var"], ora["dlnl"]))
    assert max(err["depth"], err["var"], err["dlnl"]) <= FP64_TOL, err
