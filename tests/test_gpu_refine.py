"""GPU parity of nu_periodic_refine: the exact fit of a periodic transit
column (Sect. 2.4 read as one Eq. ls over the whole curve), against the
oracle's dense and semiseparable fits."""
import numpy as np
import pytest

from oracle import gp, linear, periodic, refine, semisep
from paper_2402_06835_gb300 import synth
from parity import FP64_TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def cu(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def errors(g, o):
    """Relative errors of (depth, var, dlnl, snr); NaN at the same places."""
    nan_g = np.isnan(g["depth"])
    nan_o = np.isnan(o["depth"])
    assert np.array_equal(nan_g, nan_o), (np.flatnonzero(nan_g ^ nan_o))
    for k in ("var", "dlnl", "snr"):
        assert np.array_equal(np.isnan(g[k]), nan_o)
    ok = ~nan_o
    so = np.sqrt(o["var"][ok])
    return dict(
        depth=float((np.abs(g["depth"][ok] - o["depth"][ok])
                     / np.maximum(np.abs(o["depth"][ok]), so)).max(initial=0)),
        var=float((np.abs(g["var"][ok] - o["var"][ok]) / o["var"][ok]).max(initial=0)),
        dlnl=float((np.abs(g["dlnl"][ok] - o["dlnl"][ok])
                    / np.maximum(o["dlnl"][ok], 1.0)).max(initial=0)),
        snr=float((np.abs(g["snr"][ok] - o["snr"][ok])
                   / np.maximum(np.abs(o["snr"][ok]), 1.0)).max(initial=0)),
        n=int(ok.sum()))


def gpu_refine(f, cands, Ds, kind="box", ingress=0.1):
    P = cu([c[0] for c in cands])
    T0 = cu([c[1] for c in cands])
    J = cu([c[2] for c in cands], torch.int32)
    r = api.nu_periodic_refine(f, P, T0, J, Ds, template=kind, ingress_frac=ingress)
    return {k: v.cpu().numpy() for k, v in r.items()}


def oracle_refine(model, cands, Ds, kind="box", ingress=0.1, X=None, y=None):
    nan = float("nan")
    rows = [(P, T0, Ds[j] if 0 <= j < len(Ds) else nan) for (P, T0, j) in cands]
    return refine.refine(model, rows, kind, ingress, X=X, y=y)


def candidate_set(t, n_D, rng, n_random=120):
    span = t[-1] - t[0]
    c = [(float(rng.uniform(0.15, 3.0)), float(rng.uniform(t[0] - 1.0, t[-1] + 1.0)),
          int(rng.integers(0, n_D))) for _ in range(n_random)]
    c += [
        (10.0 * span, float(t[len(t) // 3]), n_D - 1),     # one transit
        (0.125, float(t[7]), 0),                           # many short windows
        (1.0e4, float(t[0]) - 5.0e3, 0),                   # no window reaches the data
        (0.73, float(t[0]) + 1e6 * 0.73, 1),               # epoch far from the data
        (0.41, float(t[0]), 0), (0.41, float(t[-1]), n_D - 1),
        (float("nan"), float(t[5]), 0), (0.5, float("inf"), 0),
        (0.5, float(t[5]), -1), (0.5, float(t[5]), n_D),   # D index out of range
        (-0.5, float(t[5]), 0), (0.0, float(t[5]), 0),
        (0.05, float(t[5]), n_D - 1),                      # 2 D > P
    ]
    return c


@pytest.mark.parametrize("kind", ["box", "trapezoid", "limb_quad"])
@pytest.mark.parametrize("gap", [None, 400])
def test_refine_matches_dense_oracle(kind, gap):
    lc = synth.small_curve(n=2200, seed=3, p_rot=1.3, sigma=4e-3, sigma_w=1e-3, gap=gap,
                           inject=(3e-3, 1.0 / 24.0, 0.41))
    Ds = np.array([0.03, 1.0 / 24.0, 0.055])
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    cands = candidate_set(lc.t, len(Ds), np.random.default_rng(21))
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    g = gpu_refine(f, cands, Ds, kind, 0.3)
    o = oracle_refine(model, cands, Ds, kind, 0.3)
    err = errors(g, o)
    print(f"refine {kind} gap={gap}: {err}")
    assert err["n"] >= 110
    assert max(err["depth"], err["var"], err["dlnl"], err["snr"]) <= FP64_TOL, err


def test_refine_of_the_search_candidates():
    """The oracle's periodic search picks (P, T0, D) at its best periods; both
    sides refine those.  Also reports how far Eq. result's Q (independent
    transits) is from the exact fit's SNR at full covariance."""
    lc = synth.small_curve(n=2200, seed=3, p_rot=1.3, sigma=4e-3, sigma_w=1e-3,
                           inject=(3e-3, 1.0 / 24.0, 0.41))
    Ds = np.array([0.03, 1.0 / 24.0, 0.055])
    periods = np.linspace(0.3, 0.9, 400)
    dt = periodic.median_spacing(lc.t)
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    ora = linear.linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X, lc.t, Ds, model=model)
    res = periodic.periodic_search(lc.t, ora["depth"], ora["var"], ora["dlnl"], periods, dt)
    Q = np.where(np.isfinite(res["Q"]), res["Q"], -np.inf)
    top = np.argsort(-Q)[:16]
    cands = [(float(periods[i]), float(res["T0"][i]), int(res["D_idx"][i])) for i in top]
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    g = gpu_refine(f, cands, Ds)
    o = oracle_refine(model, cands, Ds)
    err = errors(g, o)
    assert max(err["depth"], err["var"], err["dlnl"], err["snr"]) <= FP64_TOL, err
    best = top[0]
    assert abs(periods[best] - 0.41) < 0.01
    rel = abs(g["snr"][0] - Q[best]) / Q[best]
    print(f"best P {periods[best]:.4f}: Q(Eq. result) {Q[best]:.3f}, exact snr "
          f"{g['snr'][0]:.3f} (rel diff {rel:.3%}); errors {err}")
    assert g["snr"][0] > 0.5 * Q[best]


def test_refine_sector_19440_against_semiseparable_oracle():
    """Full-size sector (19 440 samples, mid-sector gap): sampled candidates
    against the O(N) semiseparable oracle."""
    w = synth.sector_19440()
    lc = w.curves[0]
    Ds = w.durations
    rng = np.random.default_rng(5)
    cands = [(float(rng.uniform(0.2, 13.5)), float(rng.uniform(lc.t[0], lc.t[-1])),
              int(rng.integers(0, len(Ds)))) for _ in range(10)]
    cands += [(3.1, float(lc.t[0]) + 0.37, 6), (0.2, float(lc.t[3]), 0),
              (13.5, float(lc.t[-1]), len(Ds) - 1)]
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    g = gpu_refine(f, cands, Ds)
    ss = semisep.Semisep(lc.t, lc.diag_var, lc.terms)
    o = oracle_refine(ss, cands, Ds, X=lc.X, y=lc.y)
    err = errors(g, o)
    print(f"refine sector_19440: {err}")
    assert err["n"] == len(cands)
    assert max(err["depth"], err["var"], err["dlnl"], err["snr"]) <= FP64_TOL, err


def test_refine_rejects_bad_arguments():
    lc = synth.small_curve(n=300, seed=2)
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    P, T0, J = cu([0.5]), cu([lc.t[3]]), cu([0], torch.int32)
    with pytest.raises(api.NuanceError):
        api.nu_periodic_refine(f, P, T0, J, [float("nan")])
    with pytest.raises(api.NuanceError):
        api.nu_periodic_refine(f, P, T0, J, [0.05], template="trapezoid", ingress_frac=0.7)
    with pytest.raises(api.NuanceError):
        api.nu_periodic_refine(f, P[:0], T0[:0], J[:0], [0.05])
    with pytest.raises(api.NuanceError):
        api.nu_periodic_refine(f, P, T0, J, [])


@pytest.mark.parametrize("terms_case", ["sho", "rotation_exp", "two_rotations"])
def test_refine_other_state_sizes(terms_case):
    """State dimensions J = 2, 6 and 8 (the segment maps, the block tables and
    the warp walk for every block count)."""
    terms = {"sho": [(gp.SHO, (5e-3, 30.0, 2.0))],
             "rotation_exp": [(gp.ROTATION, (1e-2, 0.5, 5.0, 0.0, 0.5)), (gp.EXP, (2e-3, 0.08))],
             "two_rotations": [(gp.ROTATION, (1e-2, 0.5, 5.0, 0.0, 0.5)),
                               (gp.ROTATION, (5e-3, 2.3, 3.0, 0.5, 0.3))]}[terms_case]
    lc = synth.small_curve(n=1500, seed=31, gap=200)
    Ds = np.array([0.03, 0.06])
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, terms, lc.X)
    cands = candidate_set(lc.t, len(Ds), np.random.default_rng(3), n_random=40)
    f = api.nu_gp_factor(cu(lc.t), cu(lc.diag_var), terms, cu(lc.X), cu(lc.y))
    g = gpu_refine(f, cands, Ds)
    o = oracle_refine(model, cands, Ds)
    err = errors(g, o)
    print(f"refine {terms_case}: {err}")
    assert max(err["depth"], err["var"], err["dlnl"], err["snr"]) <= FP64_TOL, err
