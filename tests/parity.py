"""Comparison helpers for the GPU-vs-oracle parity tests.

Error norms (most templates have a depth near zero, so a plain relative error
is meaningless):
  depth: |d - d_or| / max(|d_or|, sqrt(var_or))
  var:   |v - v_or| / v_or
  gain:  |g - g_or| / max(g_or, 1)
NaN must appear at the same places on both sides.

The fold's per-period outputs are compared at the argmax cell: ln P and Q,
and the combined depth Delta (norm |D - D_or| / max(|D_or|, sigma_or)) and its
sigma (relative) of Eq. sigma_delta.
"""
import numpy as np

FP64_TOL = 1e-9          # FP64 mode: depth, variance and gain
MIXED_DEPTH_TOL = 1e-4   # mixed mode: depth
MIXED_SNR_ABS = 1e-3     # mixed mode: absolute error on Q = Delta/sigma


def linear_errors(gpu, ora):
    d, v, l = (np.asarray(a, dtype=np.float64) for a in gpu)
    do, vo, lo = (np.asarray(a, dtype=np.float64) for a in ora)
    nan_g = np.isnan(d) | np.isnan(v) | np.isnan(l)
    nan_o = np.isnan(do) | np.isnan(vo) | np.isnan(lo)
    assert np.array_equal(nan_g, nan_o), (
        f"NaN pattern differs: gpu {nan_g.sum()} oracle {nan_o.sum()}")
    ok = ~nan_o
    so = np.sqrt(vo[ok])
    e_d = np.abs(d[ok] - do[ok]) / np.maximum(np.abs(do[ok]), so)
    e_v = np.abs(v[ok] - vo[ok]) / vo[ok]
    e_l = np.abs(l[ok] - lo[ok]) / np.maximum(lo[ok], 1.0)
    return dict(depth=float(e_d.max(initial=0.0)), var=float(e_v.max(initial=0.0)),
                dlnl=float(e_l.max(initial=0.0)), n=int(ok.sum()),
                n_nan=int(nan_o.sum()))


def phase_index(T0, t_ref, P, n_phi):
    return int(np.rint((T0 - t_ref) / P * n_phi))


def periodic_compare(gpu, ora, t0s, depth, var, dlnl, periods, dt, tol_lnp,
                     tol_q, fold_fn, max_reeval=200, q_abs=False, tol_ds=None):
    """Compare per-period results; near-ties in the argmax are checked by
    evaluating the oracle at the GPU's cell.  ln P, Q, the fold's depth and
    sigma are compared (tol_ds, default tol_lnp, on depth and sigma).
    Returns (worst lnP error, worst Q error, number of periods whose argmax
    cell differs); the worst depth and sigma errors are in
    periodic_compare.last."""
    tol_ds = tol_lnp if tol_ds is None else tol_ds
    g = {k: np.asarray(v) for k, v in gpu.items()}
    worst_l = worst_q = worst_d = worst_s = 0.0
    differ = 0
    for p, P in enumerate(periods):
        lo_, lg_ = ora["lnP"][p], g["lnP"][p]
        if not np.isfinite(lo_):
            assert not np.isfinite(lg_) and g["D_idx"][p] == -1 and g["Q"][p] == 0.0
            continue
        el = abs(lg_ - lo_) / max(1.0, abs(lo_))
        worst_l = max(worst_l, el)
        assert el <= tol_lnp, f"period {P}: lnP {lg_} vs {lo_}"
        n_phi = int(np.ceil(P / dt))
        jg = phase_index(g["T0"][p], t0s[0], P, n_phi)
        dg = int(g["D_idx"][p])
        if dg == ora["D_idx"][p] and jg == ora["phase_idx"][p]:
            q_o, d_o, s_o = ora["Q"][p], ora["depth"][p], ora["sigma"][p]
        else:
            differ += 1
            assert differ <= max_reeval, "too many argmax differences"
            f = fold_fn(t0s, depth, var, dlnl, P, dt)
            l_cell = f["lnP"][dg, jg]
            assert abs(l_cell - lo_) / max(1.0, abs(lo_)) <= tol_lnp, (
                f"period {P}: GPU cell ({dg},{jg}) lnP {l_cell} is not a tie of {lo_}")
            d_o, s_o = f["depth"][dg, jg], f["sigma"][dg, jg]
            q_o = d_o / s_o
        eq = abs(g["Q"][p] - q_o) / (1.0 if q_abs else max(1.0, abs(q_o)))
        worst_q = max(worst_q, eq)
        assert eq <= tol_q, f"period {P}: Q {g['Q'][p]} vs oracle {q_o}"
        if "depth" in g and "sigma" in g:
            ed = abs(g["depth"][p] - d_o) / max(abs(d_o), s_o)
            es = abs(g["sigma"][p] - s_o) / s_o
            worst_d, worst_s = max(worst_d, ed), max(worst_s, es)
            assert ed <= tol_ds, f"period {P}: depth {g['depth'][p]} vs oracle {d_o}"
            assert es <= tol_ds, f"period {P}: sigma {g['sigma'][p]} vs oracle {s_o}"
    periodic_compare.last = dict(lnP=worst_l, Q=worst_q, depth=worst_d, sigma=worst_s,
                                 ties=differ)
    return worst_l, worst_q, differ


periodic_compare.last = {}
