"""Exact periodic-template fit of a candidate (test only).

Sect. 2.4 defines Q(P) as the SNR Delta/sigma of a periodic transit of
period P, epoch T0 = phi0 P and duration D.  The periodic search obtains
Delta and sigma from the single events combined with Eq. result, which
treats the transits as independent (Sect. 2.3 states that approximation).
The other reading of Sect. 2.4 is the fit itself: Eq. ls with the design
matrix X' = [X, m_P], whose last column m_P is the periodic box of unit depth,
solved once over the whole light curve at full covariance.  This module
computes that fit for given candidates (P, T0, D); comparing its Q with the
fold's measures the independence approximation.

Definitions (readings listed with the design):

* m_P(t) = sum over all integers n of m(t; T0 + n P, D), where m is the
  single-transit template of ``oracle.linear.template`` (box, trapezoid or
  limb-darkened, the same half-open window) and each centre T0 + n P is
  evaluated in FP64 as written (the product n P rounded, then the sum);
* the windows must not overlap: a candidate needs 0 < 2 D <= P; a candidate
  that is not finite, breaks that, or whose template has no non-zero sample,
  gets NaN for depth, var, dlnl and snr;
* depth, var and dlnl are those of Eq. ls and Eq. linear_search_ll
  (``DenseModel.fit_templates`` or, for long curves, ``Semisep.fit_templates``)
  and snr = depth / sqrt(var).

Nothing here shares code with the CUDA sources.
"""
from __future__ import annotations

import math

import numpy as np

from .linear import template


def valid_candidate(P, T0, D):
    """The candidate conditions above (finite, D > 0, 2 D <= P)."""
    return (math.isfinite(P) and math.isfinite(T0) and math.isfinite(D)
            and D > 0.0 and 2.0 * D <= P)


def periodic_template(t, P, T0, D, kind="box", ingress_frac=0.1, ld=(0.4, 0.25)):
    """m_P(t): the single template repeated at every T0 + n P.

    Every n whose window can reach [t_min, t_max] is summed; the range is
    widened by one period on each side so that rounding of the estimate
    cannot drop a window.
    """
    t = np.asarray(t, dtype=np.float64)
    if not valid_candidate(P, T0, D):
        raise ValueError("candidate needs finite P, T0, D with 0 < 2 D <= P")
    n_lo = math.floor((t[0] - T0 - D) / P) - 1
    n_hi = math.ceil((t[-1] - T0 + D) / P) + 1
    m = np.zeros_like(t)
    for n in range(n_lo, n_hi + 1):
        m += template(t, T0 + float(n) * P, D, kind, ingress_frac, ld)
    return m


def refine(model, candidates, kind="box", ingress_frac=0.1, X=None, y=None,
           ld=(0.4, 0.25)):
    """Eq. ls with the periodic template for each (P, T0, D) of candidates.

    model is an ``oracle.linear.DenseModel`` or an ``oracle.semisep.Semisep``
    (the latter needs X and y).  Returns dict of (n_cand,) arrays depth, var,
    dlnl, snr.
    """
    cands = [tuple(float(v) for v in c) for c in candidates]
    nc = len(cands)
    out = {k: np.full(nc, np.nan) for k in ("depth", "var", "dlnl", "snr")}
    ok = [i for i, (P, T0, D) in enumerate(cands) if valid_candidate(P, T0, D)]
    if not ok:
        return out
    M = np.stack([periodic_template(model.t, *cands[i], kind, ingress_frac, ld)
                  for i in ok], axis=1)
    if X is None:
        d, v, l = model.fit_templates(M)
    else:
        d, v, l = model.fit_templates(X, np.asarray(y, dtype=np.float64), M)
    for slot, i in enumerate(ok):
        out["depth"][i] = d[slot]
        out["var"][i] = v[slot]
        out["dlnl"][i] = l[slot]
        out["snr"][i] = d[slot] / np.sqrt(v[slot])
    return out
