"""Periodic search oracle: fold single events into SNR(P) (test only).

Follows Sect. 2.3 ("The periodic search"), Sect. 2.4 ("The transit-search
periodogram") and Appendix B:

* for a period P, a duration D and a phase, the K epochs of a periodic
  transit are combined with Eq. result,
      ln P = sum_k ln L_k - 1/2 sum_k [ ln sigma_k^2 - ln(sigma^2 + sigma_k^2)
                                        + (Delta_k - Delta)^2 / (sigma_k^2 + sigma^2) ],
  using the biased (all-k) estimates of Eq. sigma_delta,
      1/sigma^2 = sum_k 1/sigma_k^2,  Delta = sigma^2 sum_k Delta_k / sigma_k^2;
* the single-event values are interpolated from the epoch grid onto a common
  grid of phases (Sect. 2.3, "instead of nearest neighbours");
* (phi0, D) is the argmax of ln P over phases and durations (Eq. phi0) and
  Q(P) = Delta / sigma at that cell (Sect. 2.4).

Readings where the text is silent or ambiguous (listed with the design):
* ln L_k is taken as the log-likelihood gain of the single event over the
  transit-free model, so that the number of combined points does not enter
  (the normalisation caveat of Sect. 2.4);
* phases phi_j = j / n_phi with n_phi = ceil(P / dt), dt the median epoch
  spacing unless given; the reference epoch is the first grid epoch (the
  paper's "T_0 = 0"), epochs T = T_ref + (phi_j + k) P for every k >= 0 with
  T <= last grid epoch; the reported epoch is T_ref + phi0 P;
* interpolation is linear in time between the two bracketing grid epochs
  (the largest i with t0_i <= T, and i + 1) of the stored triple
  (Delta, sigma = sqrt(var), ln L gain); an epoch is left out when it has no
  right neighbour, when the two grid epochs are more than gap_factor * dt
  apart, or when either node holds a non-finite value or var <= 0;
* a cell with no epoch has ln P = -inf and is never selected; the argmax is
  the first maximum in duration-major then phase order; a period with no
  valid cell reports Q = 0, ln P = -inf and duration index -1.
"""
from __future__ import annotations

import numpy as np


def median_spacing(t0s):
    return float(np.median(np.diff(np.asarray(t0s, dtype=np.float64))))


def epoch_penalty(dk, sk2, delta, s2):
    """One term of the second sum of Eq. result."""
    return np.log(sk2) - np.log(s2 + sk2) + (dk - delta) ** 2 / (sk2 + s2)


def combine(dk, sk2, lk):
    """Eq. result with Eq. sigma_delta for 1-D arrays of K single events.

    Returns (lnP, Delta, sigma).  K = 0 gives (-inf, nan, nan).
    """
    dk = np.asarray(dk, dtype=np.float64)
    sk2 = np.asarray(sk2, dtype=np.float64)
    lk = np.asarray(lk, dtype=np.float64)
    if dk.size == 0:
        return -np.inf, np.nan, np.nan
    inv_s2 = np.sum(1.0 / sk2)
    s2 = 1.0 / inv_s2
    delta = s2 * np.sum(dk / sk2)
    lnp = np.sum(lk) - 0.5 * np.sum(epoch_penalty(dk, sk2, delta, s2))
    return lnp, delta, np.sqrt(s2)


def interpolate(t0s, depth, var, dlnl, T, dt, gap_factor=1.5):
    """Linear interpolation of the single-event grid at epochs T (any shape).

    depth/var/dlnl are (n_D, n_t0).  Returns (valid, d_k, s_k, l_k) where
    valid has T's shape and the values have shape (n_D,) + T.shape.
    """
    t0s = np.asarray(t0s, dtype=np.float64)
    n = len(t0s)
    T = np.asarray(T, dtype=np.float64)
    i = np.searchsorted(t0s, T, side="right") - 1
    inside = (i >= 0) & (i <= n - 2)
    ic = np.clip(i, 0, n - 2)
    ta = t0s[ic]
    tb = t0s[ic + 1]
    inside &= (tb - ta) <= gap_factor * dt
    w = (T - ta) / (tb - ta)
    sig = np.sqrt(np.where(var > 0, var, np.nan))
    da, db = depth[:, ic], depth[:, ic + 1]
    sa, sb = sig[:, ic], sig[:, ic + 1]
    la, lb = dlnl[:, ic], dlnl[:, ic + 1]
    d_k = (1.0 - w) * da + w * db
    s_k = (1.0 - w) * sa + w * sb
    l_k = (1.0 - w) * la + w * lb
    finite = (np.isfinite(da) & np.isfinite(db) & np.isfinite(sa)
              & np.isfinite(sb) & np.isfinite(la) & np.isfinite(lb))
    valid = inside[None] & finite
    return valid, d_k, s_k, l_k


def epochs(P, n_phi, t_ref, t_last):
    """T[j, k] = t_ref + (j/n_phi + k) P and the mask T <= t_last."""
    kmax = int(np.floor((t_last - t_ref) / P)) + 2
    phi = np.arange(n_phi, dtype=np.float64) / n_phi
    k = np.arange(kmax, dtype=np.float64)
    T = t_ref + (phi[:, None] + k[None, :]) * P
    return T, T <= t_last


def fold_period(t0s, depth, var, dlnl, P, dt, gap_factor=1.5):
    """ln P, Delta, sigma and K for every (duration, phase) cell at period P."""
    t0s = np.asarray(t0s, dtype=np.float64)
    n_phi = int(np.ceil(P / dt))
    T, in_range = epochs(P, n_phi, t0s[0], t0s[-1])
    valid, d_k, s_k, l_k = interpolate(t0s, depth, var, dlnl, T, dt,
                                       gap_factor)
    m = valid & in_range[None]
    sk2 = np.where(m, s_k * s_k, 1.0)
    dk = np.where(m, d_k, 0.0)
    lk = np.where(m, l_k, 0.0)
    K = m.sum(axis=-1)
    inv_s2 = np.where(m, 1.0 / sk2, 0.0).sum(axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        s2 = 1.0 / inv_s2
        delta = s2 * np.where(m, dk / sk2, 0.0).sum(axis=-1)
        pen = np.where(m, epoch_penalty(dk, sk2, delta[..., None],
                                        s2[..., None]), 0.0).sum(axis=-1)
        lnp = lk.sum(axis=-1) - 0.5 * pen
    lnp = np.where(K > 0, lnp, -np.inf)
    return dict(lnP=lnp, depth=np.where(K > 0, delta, np.nan),
                sigma=np.where(K > 0, np.sqrt(s2), np.nan), K=K, n_phi=n_phi)


def periodic_search(t0s, depth, var, dlnl, periods, dt=None, gap_factor=1.5):
    """Q(P) periodogram (Sect. 2.4) with the best cell of Eq. phi0 per P."""
    t0s = np.asarray(t0s, dtype=np.float64)
    if dt is None or dt <= 0:
        dt = median_spacing(t0s)
    nP = len(periods)
    res = {k: np.full(nP, np.nan) for k in ("Q", "T0", "depth", "sigma", "lnP")}
    res["D_idx"] = np.full(nP, -1, dtype=np.int64)
    res["phase_idx"] = np.full(nP, -1, dtype=np.int64)
    for p, P in enumerate(np.asarray(periods, dtype=np.float64)):
        f = fold_period(t0s, depth, var, dlnl, P, dt, gap_factor)
        score = np.where(np.isfinite(f["lnP"]), f["lnP"], -np.inf)
        if not np.any(np.isfinite(score)):
            res["Q"][p] = 0.0
            res["lnP"][p] = -np.inf
            continue
        flat = int(np.argmax(score))            # first max, duration-major
        d, j = divmod(flat, score.shape[1])
        res["D_idx"][p] = d
        res["phase_idx"][p] = j
        res["lnP"][p] = f["lnP"][d, j]
        res["depth"][p] = f["depth"][d, j]
        res["sigma"][p] = f["sigma"][d, j]
        res["Q"][p] = f["depth"][d, j] / f["sigma"][d, j]
        res["T0"][p] = t0s[0] + (j / f["n_phi"]) * P
    res["dt"] = dt
    return res


def best(res, periods):
    """Best candidate: first maximum of Q over the periods (Sect. 2.4)."""
    q = np.where(np.isfinite(res["Q"]), res["Q"], -np.inf)
    p = int(np.argmax(q))
    return dict(period=float(periods[p]), T0=float(res["T0"][p]),
                D_idx=int(res["D_idx"][p]), depth=float(res["depth"][p]),
                sigma=float(res["sigma"][p]), Q=float(res["Q"][p]), index=p)


def mask_transits(t0s, depth, var, dlnl, P, T0, half_width):
    """Masking of a found candidate before the next search (Sect. 2.5, and
    the TOI-540 comparison of Sect. 3.3: trial epochs in windows of width
    2 D centred on the detected transits are masked in the linear-search
    products).  Entries of every duration whose epoch lies within
    half_width of T0 + n P (n the nearest integer, each operation rounded
    once in FP64) become NaN.  Returns masked copies and the epoch mask."""
    t0s = np.asarray(t0s, dtype=np.float64)
    n = np.rint((t0s - T0) / P)
    dist = np.abs(t0s - (T0 + n * P))
    m = dist < half_width
    out = []
    for a in (depth, var, dlnl):
        b = np.array(a, copy=True)
        b[:, m] = np.nan
        out.append(b)
    return out[0], out[1], out[2], m


def rotation_alias_keep(periods, P_star, tol=0.02, symmetric=False):
    """Sect. 3's exclusion of the rotation period's aliases from the grid.

    With dP = P / P_star a period is removed when |dP - ceil(dP)| < tol (the
    printed criterion), or, symmetric, when |dP - rint(dP)| < tol (the
    wording "less than 2 % from an integer").  Returns the boolean keep mask.
    """
    P = np.asarray(periods, dtype=np.float64)
    dP = P / P_star
    ref = np.rint(dP) if symmetric else np.ceil(dP)
    with np.errstate(invalid="ignore"):
        drop = np.abs(dP - ref) < tol
    return ~drop
