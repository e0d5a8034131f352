"""Comparison helpers for the GPU-vs-oracle parity tests.

Error norms (most templates have a depth near zero, so a plain relative error
is meaningless):
  depth: |d - d_or| / max(|d_or|, sqrt(var_or))
  var:   |v - v_or| / v_or
  gain:  |g - g_or| / max(g_or, 1)
NaN must appear at the same places on both sides.
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
                     tol_q, fold_fn, max_reeval=200, q_abs=False):
    """Compare per-period results; near-ties in the argmax are checked by
    evaluating the oracle at the GPU's cell.  Returns (worst lnP error,
    worst Q error, number of periods whose argmax cell differs)."""
    g = {k: np.asarray(v) for k, v in gpu.items()}
    worst_l = worst_q = 0.0
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
            eq = abs(g["Q"][p] - ora["Q"][p]) / (1.0 if q_abs else max(1.0, abs(ora["Q"][p])))
        else:
            differ += 1
            assert differ <= max_reeval, "too many argmax differences"
            f = fold_fn(t0s, depth, var, dlnl, P, dt)
            l_cell = f["lnP"][dg, jg]
            assert abs(l_cell - lo_) / max(1.0, abs(lo_)) <= tol_lnp, (
                f"period {P}: GPU cell ({dg},{jg}) lnP {l_cell} is not a tie of {lo_}")
            q_cell = f["depth"][dg, jg] / f["sigma"][dg, jg]
            eq = abs(g["Q"][p] - q_cell) / (1.0 if q_abs else max(1.0, abs(q_cell)))
        worst_q = max(worst_q, eq)
        assert eq <= tol_q, f"period {P}: Q {g['Q'][p]} vs oracle"
    return worst_l, worst_q, differ
