"""Sequential FP64 celerite reference for long light curves (test only).

The dense oracle needs the N x N covariance, which does not fit for the
seven-sector light curve (N = 136 080, 148 GB).  This module evaluates the
same linear search (Sect. 2.2, Eq. ls and Eq. linear_search_ll) without the
dense matrix, through the semiseparable Cholesky factorisation of the
celerite method that the paper's GP library implements (Foreman-Mackey et al.
2017, AJ 154, 220, Sect. 5):

  k(tau) = sum_j e^{-c_j tau} (a_j cos(d_j tau) + b_j sin(d_j tau)),
  for the SHO of Appendix A with Q > 1/2: a = sigma^2, b = sigma^2/g,
  c = omega/(2Q), d = g omega/(2Q), g = sqrt(4Q^2 - 1);
  for an exponential term: a = sigma^2, c = 1/ell, b = d = 0;
  U_n = [a cos(d t_n) + b sin(d t_n), a sin(d t_n) - b cos(d t_n)],
  V_n = [cos(d t_n), sin(d t_n)], phi_n = e^{-c (t_n - t_{n-1})},
  A_n = diag_var_n + sum_j a_j,
  S_n = diag(phi_n) (S_{n-1} + D_{n-1} W_{n-1} W_{n-1}^T) diag(phi_n),
  D_n = A_n - U_n^T S_n U_n,  W_n = (V_n - S_n U_n) / D_n,
  forward solve of L z = y:   f_n = phi_n (f_{n-1} + W_{n-1} z_{n-1}),
                              z_n = y_n - U_n^T f_n.

The GLS of every requested template is then solved from the forward
innovations e = L^-1 [X, y, m] weighted by 1/D (so that a^T Sigma^-1 b =
e_a^T D^-1 e_b), with the chi-square of Eq. linear_search_ll from the
whitened residual.  Every recursion is a plain Python loop over the samples
(numpy only for the small per-sample vectors); the reference is pinned to
``oracle.linear`` on sizes where both run.
"""
from __future__ import annotations

import numpy as np

from . import gp
from .linear import LOG2PI, template


def celerite_terms(terms):
    """(a, b, c, d) per celerite term for the SHO (Q > 1/2) and EXP kinds."""
    out = []
    for kind, p in terms:
        if kind == gp.SHO:
            shos = [tuple(p[:3])]
        elif kind == gp.ROTATION:
            shos = gp.rotation_sho_params(*p[:5])
        elif kind == gp.EXP:
            out.append((p[0] ** 2, 0.0, 1.0 / p[1], 0.0))
            continue
        else:
            raise ValueError(kind)
        for sigma, omega, Q in shos:
            if not Q > 0.5:
                raise ValueError("this reference covers Q > 1/2 only")
            g = np.sqrt(4.0 * Q * Q - 1.0)
            out.append((sigma * sigma, sigma * sigma / g, omega / (2.0 * Q),
                        g * omega / (2.0 * Q)))
    return out


class Semisep:
    """Celerite factorisation Sigma = L diag(D) L^T of one light curve."""

    def __init__(self, t, diag_var, terms):
        t = np.asarray(t, dtype=np.float64)
        self.t = t
        self.N = len(t)
        coeffs = celerite_terms(terms)
        cols_U, cols_V, cs = [], [], []
        for a, b, c, d in coeffs:
            if d == 0.0 and b == 0.0:
                cols_U.append(np.full(self.N, a))
                cols_V.append(np.ones(self.N))
                cs.append(c)
            else:
                cd, sd = np.cos(d * t), np.sin(d * t)
                cols_U += [a * cd + b * sd, a * sd - b * cd]
                cols_V += [cd, sd]
                cs += [c, c]
        self.U = np.stack(cols_U, axis=1)
        self.V = np.stack(cols_V, axis=1)
        c = np.array(cs)
        dt = np.diff(t, prepend=t[0])
        self.phi = np.exp(-c[None, :] * dt[:, None])
        A = np.asarray(diag_var, dtype=np.float64) + sum(a for a, _, _, _ in coeffs)
        R = self.U.shape[1]
        self.D = np.empty(self.N)
        self.W = np.empty((self.N, R))
        S = np.zeros((R, R))
        for n in range(self.N):
            if n > 0:
                S = self.phi[n][:, None] * (S + self.D[n - 1] * np.outer(self.W[n - 1],
                                                                         self.W[n - 1])) \
                    * self.phi[n][None, :]
            Un = self.U[n]
            SU = S @ Un
            self.D[n] = A[n] - Un @ SU
            self.W[n] = (self.V[n] - SU) / self.D[n]
        self.logdet = float(np.sum(np.log(self.D)))

    def innovations(self, Y):
        """e = L^-1 Y for the columns of Y (N, m)."""
        Y = np.asarray(Y, dtype=np.float64).reshape(self.N, -1)
        E = np.empty_like(Y)
        f = np.zeros((self.U.shape[1], Y.shape[1]))
        for n in range(self.N):
            if n > 0:
                f = self.phi[n][:, None] * (f + np.outer(self.W[n - 1], E[n - 1]))
            E[n] = Y[n] - self.U[n] @ f
        return E

    def fit_templates(self, X, y, M):
        """Eq. ls + Eq. linear_search_ll for templates M (N, B) given X, y."""
        X = np.asarray(X, dtype=np.float64).reshape(self.N, -1)
        k = X.shape[1]
        M = np.asarray(M, dtype=np.float64).reshape(self.N, -1)
        E = self.innovations(np.concatenate([X, y[:, None], M], axis=1))
        w = 1.0 / self.D
        eX, ey, eM = E[:, :k], E[:, k], E[:, k + 1:]
        # null model
        if k:
            A0 = eX.T @ (w[:, None] * eX)
            w0 = np.linalg.solve(A0, eX.T @ (w * ey))
            r0 = ey - eX @ w0
        else:
            r0 = ey
        chi0 = float(r0 @ (w * r0))
        depth = np.full(M.shape[1], np.nan)
        var = np.full(M.shape[1], np.nan)
        dlnl = np.full(M.shape[1], np.nan)
        for b in range(M.shape[1]):
            if not np.any(M[:, b] != 0.0):
                continue
            Ep = np.concatenate([eX, eM[:, b:b + 1]], axis=1)
            G = Ep.T @ (w[:, None] * Ep)
            cov = np.linalg.inv(G)
            wt = cov @ (Ep.T @ (w * ey))
            r = ey - Ep @ wt
            chi = float(r @ (w * r))
            depth[b] = wt[-1]
            var[b] = cov[-1, -1]
            dlnl[b] = 0.5 * (chi0 - chi)
        self.chi2_null = chi0
        self.lnL_null = -0.5 * chi0 - 0.5 * self.logdet - 0.5 * self.N * LOG2PI
        return depth, var, dlnl


def sampled_linear_search(t, y, diag_var, terms, X, Ds, pairs, kind="box",
                          ingress_frac=0.1, model=None, ld=(0.4, 0.25)):
    """Templates for (duration index, t0 index) pairs with t0s = t."""
    if model is None:
        model = Semisep(t, diag_var, terms)
    M = np.stack([template(model.t, t[i], Ds[j], kind, ingress_frac, ld) for (j, i) in pairs],
                 axis=1)
    d, v, l = model.fit_templates(X, np.asarray(y, dtype=np.float64), M)
    return d, v, l, model
