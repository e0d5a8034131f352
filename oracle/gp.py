"""Covariance of the light-curve model (oracle; test infrastructure only).

Sources:
* Appendix A ("SHO kernel"): k(tau) = sigma^2 exp(-omega tau / 2Q) times
  1 + omega tau (Q = 1/2), cosh(f omega tau/2Q) + sinh(f omega tau/2Q)/f
  (Q < 1/2, f = sqrt(1 - 4Q^2)), cos(g omega tau/2Q) + sin(g omega tau/2Q)/g
  (Q > 1/2, g = sqrt(4Q^2 - 1)), tau = |t_i - t_j|.
* Sect. 3.2 "Stellar variability kernel": the rotation kernel k1 + k2 with
  Q1 = 1/2 + Q0 + dQ, omega1 = 4 pi Q1 / (P sqrt(4 Q1^2 - 1)),
  S1 = sigma^2 / ((1 + f) omega1 Q1); Q2 = 1/2 + Q0, omega2 = 2 omega1,
  S2 = f sigma^2 / ((1 + f) omega2 Q2); and the exponential terms
  k(t, t') = sigma^2 exp(-|t - t'| / ell).
* Sect. 2.1 (Fig. 1 caption, Eq. linear_model): white noise is added to the
  diagonal of the covariance matrix.

The SHO amplitude in the S-parametrisation of Sect. 3.2 is tied to the sigma
of Appendix A by sigma^2 = S omega Q (the zero-lag value of the celerite SHO
term, Foreman-Mackey et al. 2017, AJ 154, 220).
"""
from __future__ import annotations

import numpy as np

SHO = 0
EXP = 1
ROTATION = 2


def sho_kernel(tau, sigma, omega, Q):
    """Appendix A SHO covariance at lags ``tau`` (any shape, tau >= 0)."""
    tau = np.abs(np.asarray(tau, dtype=np.float64))
    x = omega * tau / (2.0 * Q)
    env = sigma * sigma * np.exp(-x)
    if Q == 0.5:
        return env * (1.0 + omega * tau)
    if Q < 0.5:
        f = np.sqrt(1.0 - 4.0 * Q * Q)
        return env * (np.cosh(f * x) + np.sinh(f * x) / f)
    g = np.sqrt(4.0 * Q * Q - 1.0)
    return env * (np.cos(g * x) + np.sin(g * x) / g)


def exp_kernel(tau, sigma, ell):
    """Sect. 3.2 exponential term sigma^2 exp(-|tau| / ell)."""
    tau = np.abs(np.asarray(tau, dtype=np.float64))
    return sigma * sigma * np.exp(-tau / ell)


def rotation_sho_params(sigma, period, Q0, dQ, f):
    """Sect. 3.2 map from (sigma, P, Q0, dQ, f) to two SHO terms.

    Returns [(sigma_1, omega_1, Q_1), (sigma_2, omega_2, Q_2)] in the
    Appendix A parametrisation, sigma_j^2 = S_j omega_j Q_j.
    """
    Q1 = 0.5 + Q0 + dQ
    w1 = 4.0 * np.pi * Q1 / (period * np.sqrt(4.0 * Q1 * Q1 - 1.0))
    S1 = sigma * sigma / ((1.0 + f) * w1 * Q1)
    Q2 = 0.5 + Q0
    w2 = 2.0 * w1
    S2 = f * sigma * sigma / ((1.0 + f) * w2 * Q2)
    return [(np.sqrt(S1 * w1 * Q1), w1, Q1), (np.sqrt(S2 * w2 * Q2), w2, Q2)]


def kernel_function(terms):
    """Return k(tau) for a list of (kind, params) terms summed (Sect. 3.2)."""
    parts = []
    for kind, p in terms:
        if kind == SHO:
            parts.append(lambda tau, p=p: sho_kernel(tau, p[0], p[1], p[2]))
        elif kind == EXP:
            parts.append(lambda tau, p=p: exp_kernel(tau, p[0], p[1]))
        elif kind == ROTATION:
            for (s, w, q) in rotation_sho_params(*p[:5]):
                parts.append(lambda tau, s=s, w=w, q=q: sho_kernel(tau, s, w, q))
        else:
            raise ValueError(f"unknown term kind {kind}")

    def k(tau):
        out = np.zeros_like(np.asarray(tau, dtype=np.float64))
        for part in parts:
            out = out + part(tau)
        return out

    return k


def covariance(t, diag_var, terms):
    """Dense Sigma_ab = k(|t_a - t_b|) + delta_ab diag_var_a (Sect. 2.1)."""
    t = np.asarray(t, dtype=np.float64)
    tau = np.abs(t[:, None] - t[None, :])
    S = kernel_function(terms)(tau)
    S[np.diag_indices_from(S)] += np.asarray(diag_var, dtype=np.float64)
    return S
