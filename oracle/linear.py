"""Linear search oracle: one dense GLS fit per (epoch, duration) (test only).

Follows Sect. 2.2 ("The linear search") and Sect. 2.1 ("The approach"):

* the design matrix of a template is X' = [X, m(t0, D)], the transit being its
  last column (Eq. linear_model, Sect. 2.1);
* the weights are the generalised least-squares solution
  w = (X'^T Sigma^-1 X')^-1 X'^T Sigma^-1 f with covariance
  (X'^T Sigma^-1 X')^-1 (Eq. ls); the depth is the last weight and its
  variance the last diagonal entry of that covariance (the "uncertainties
  sigma" that Sect. 2.2 stores for the periodic search);
* the log-likelihood is Eq. linear_search_ll evaluated at those weights;
  the returned gain is that log-likelihood minus the same quantity for the
  model without the transit column.

Readings where the paper is not explicit (they are listed with the design):
the box template is -1 inside the window and 0 outside, so that a dip has a
positive depth; a sample belongs to the window when t0 - D/2 <= t < t0 + D/2
(half-open, evaluated in FP64 exactly as written); the trapezoid (not in the
paper) has total width D, linear ingress and egress of width ingress_frac*D
and a flat bottom of -1; the limb-darkened template (Sect. 4.4 names
limb-darkened transits as a base model to come) is the small-planet,
central-transit profile under the quadratic law on the same window.

How it is evaluated: Sigma is formed densely (``oracle.gp.covariance``) and
factored once, Sigma = C C^T (LAPACK Cholesky).  Every column is whitened by
C^-1 (triangular solves), after which Eq. ls is an ordinary least-squares
problem A w = y~ with A = C^-1 X'; it is solved through a QR factorisation of
A (so that X'^T Sigma^-1 X' = R^T R is never formed and its condition number
is not squared), and the chi-square of Eq. linear_search_ll is the squared
norm of the whitened residual.  No blocking, recursion or closed form of the
CUDA path is used.

For a whole grid of box templates on a long light curve (tens of thousands of
samples), whitening every template costs O(N^2) each; ``box_grid`` takes the
other dense route: Sigma^-1 once (N^3), then per template the window's block
sum of Sigma^-1 and the elimination of the transit column from the normal
equations (O(L^2) per template).  It is pinned to the brute force, the
weighted-BLS closed form, noiseless recovery and the QR route.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import gp

LOG2PI = np.log(2.0 * np.pi)


def box_template(t, t0, D):
    """Normalised box: -1 for t0 - D/2 <= t < t0 + D/2, else 0."""
    t = np.asarray(t, dtype=np.float64)
    lo = t0 - D * 0.5
    hi = t0 + D * 0.5
    return np.where((t >= lo) & (t < hi), -1.0, 0.0)


def trapezoid_template(t, t0, D, ingress_frac):
    """Trapezoid of total width D, ramps of ingress_frac*D, bottom -1."""
    t = np.asarray(t, dtype=np.float64)
    half = D * 0.5
    ramp = ingress_frac * D
    depth = (half - np.abs(t - t0)) / ramp
    inside = (t >= t0 - half) & (t < t0 + half)
    return np.where(inside, -np.clip(depth, 0.0, 1.0), 0.0)


def limb_quad_template(t, t0, D, u1, u2):
    """Limb-darkened transit as base model (the prospect of Sect. 4.4).

    Small-planet limit of a central transit (Mandel & Agol 2002, ApJ 580,
    L171, Sect. 5): the planet at projected distance r = 2 (t - t0) / D stellar
    radii blocks flux in proportion to the local intensity, here the quadratic
    law I(mu) = 1 - u1 (1 - mu) - u2 (1 - mu)^2 with mu = sqrt(1 - r^2).  The
    template is -I on the box's window (-1 at the centre), 0 outside.
    """
    t = np.asarray(t, dtype=np.float64)
    inside = (t >= t0 - D * 0.5) & (t < t0 + D * 0.5)
    r = np.where(inside, 2.0 * (t - t0) / D, 0.0)
    mu = np.sqrt(1.0 - r * r)
    x = 1.0 - mu
    intensity = 1.0 - u1 * x - u2 * x * x
    return np.where(inside, -intensity, 0.0)


def template(t, t0, D, kind="box", ingress_frac=0.1, ld=(0.4, 0.25)):
    if kind == "box":
        return box_template(t, t0, D)
    if kind == "trapezoid":
        return trapezoid_template(t, t0, D, ingress_frac)
    if kind == "limb_quad":
        return limb_quad_template(t, t0, D, ld[0], ld[1])
    raise ValueError(kind)


class DenseModel:
    """Dense FP64 model of one light curve: Sigma, its factor and the null fit."""

    def __init__(self, t, y, diag_var, terms, X):
        self.t = np.asarray(t, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.N = len(self.t)
        X = np.asarray(X, dtype=np.float64).reshape(self.N, -1)
        self.X = X
        self.k = X.shape[1]
        Sigma = gp.covariance(self.t, diag_var, terms)
        self.C = np.linalg.cholesky(Sigma)
        del Sigma
        self.logdet = 2.0 * np.sum(np.log(np.diag(self.C)))
        self.yw = solve_triangular(self.C, self.y, lower=True)
        self.Xw = solve_triangular(self.C, X, lower=True) if self.k else X
        if self.k:
            w0, _ = _ols_qr(self.Xw[None], self.yw[None])
            r0 = self.yw - self.Xw @ w0[0]
        else:
            r0 = self.yw
        self.chi2_null = float(r0 @ r0)
        self.lnL_null = (-0.5 * self.chi2_null - 0.5 * self.logdet
                         - 0.5 * self.N * LOG2PI)

    def fit_templates(self, M):
        """Eq. ls + Eq. linear_search_ll for templates M (N, B).

        Returns (depth, var, dlnl), each (B,).  A template with no non-zero
        sample, or one that lies in the span of X, has no depth: NaN triple.
        """
        M = np.asarray(M, dtype=np.float64).reshape(self.N, -1)
        B = M.shape[1]
        Mw = solve_triangular(self.C, M, lower=True)
        A = np.empty((B, self.N, self.k + 1))
        if self.k:
            A[:, :, :self.k] = self.Xw[None]
        A[:, :, self.k] = Mw.T
        yb = np.broadcast_to(self.yw, (B, self.N))
        w, var = _ols_qr(A, yb)
        resid = yb - np.einsum("bnk,bk->bn", A, w)
        chi2 = np.einsum("bn,bn->b", resid, resid)
        lnL = -0.5 * chi2 - 0.5 * self.logdet - 0.5 * self.N * LOG2PI
        depth = w[:, -1].copy()
        dvar = var.copy()
        dlnl = lnL - self.lnL_null
        bad = ~np.any(M != 0.0, axis=0) | ~np.isfinite(dvar) | (dvar <= 0)
        depth[bad] = np.nan
        dvar[bad] = np.nan
        dlnl[bad] = np.nan
        return depth, dvar, dlnl

    def lnL_full(self, dlnl):
        """Eq. linear_search_ll value from a gain (adds the null model back)."""
        return np.asarray(dlnl) + self.lnL_null


def _ols_qr(A, y):
    """Batched least squares via QR: returns (w, last diagonal of (A^T A)^-1)."""
    Q, R = np.linalg.qr(A)                         # A = Q R, R upper (B, p, p)
    qty = np.einsum("bnp,bn->bp", Q, y)
    p = R.shape[-1]
    w = np.empty(qty.shape)
    var = np.full(A.shape[0], np.nan)
    diagR = np.abs(np.diagonal(R, axis1=1, axis2=2))
    scale = np.max(diagR, axis=1)
    ok = np.min(diagR, axis=1) > 1e-13 * np.maximum(scale, 1e-300)
    for b in range(A.shape[0]):
        if not ok[b]:
            w[b] = np.nan
            continue
        w[b] = solve_triangular(R[b], qty[b], lower=False)
        # (A^T A)^-1 = R^-1 R^-T; its last diagonal entry is 1 / R[p-1, p-1]^2
        Rinv = solve_triangular(R[b], np.eye(p), lower=False)
        var[b] = Rinv[p - 1] @ Rinv[p - 1]
    return w, var


def linear_search(t, y, diag_var, terms, X, t0s, Ds, kind="box",
                  ingress_frac=0.1, chunk=256, model=None, ld=(0.4, 0.25)):
    """Sect. 2.2 linear search on the (t0s x Ds) grid.

    Returns dict with depth, var, dlnl of shape (n_D, n_t0) (duration-major),
    plus logdet and lnL_null of the template-free model.
    """
    if model is None:
        model = DenseModel(t, y, diag_var, terms, X)
    t0s = np.asarray(t0s, dtype=np.float64)
    Ds = np.asarray(Ds, dtype=np.float64)
    out = {name: np.full((len(Ds), len(t0s)), np.nan)
           for name in ("depth", "var", "dlnl")}
    for j, D in enumerate(Ds):
        for s in range(0, len(t0s), chunk):
            sl = slice(s, min(s + chunk, len(t0s)))
            M = np.stack([template(model.t, t0, D, kind, ingress_frac, ld)
                          for t0 in t0s[sl]], axis=1)
            d, v, l = model.fit_templates(M)
            out["depth"][j, sl] = d
            out["var"][j, sl] = v
            out["dlnl"][j, sl] = l
    out["logdet"] = model.logdet
    out["lnL_null"] = model.lnL_null
    return out


def sampled_linear_search(model, t0s, Ds, pairs, kind="box", ingress_frac=0.1,
                          ld=(0.4, 0.25)):
    """Templates for a list of (duration index, t0 index) pairs only."""
    M = np.stack([template(model.t, t0s[i], Ds[j], kind, ingress_frac, ld)
                  for (j, i) in pairs], axis=1)
    return model.fit_templates(M)


def box_windows(t, t0s, D):
    """Sample index range [lo, hi) of the box window of each epoch: the
    samples with t0 - D/2 <= t < t0 + D/2 (both ends evaluated in FP64 as
    written)."""
    t = np.asarray(t, dtype=np.float64)
    t0s = np.asarray(t0s, dtype=np.float64)
    lo = np.searchsorted(t, t0s - D * 0.5, side="left")
    hi = np.searchsorted(t, t0s + D * 0.5, side="left")
    return lo, hi


def box_grid(model, t0s, Ds):
    """Sect. 2.2 for the box template on a whole (t0s x Ds) grid, for light
    curves whose every template cannot be whitened one by one.

    Route (the dense alternative for long curves): Sigma^-1 is formed once
    from the Cholesky factor (LAPACK dpotri), and Eq. ls for X' = [X, m] is
    solved by eliminating the transit column (block Gaussian elimination of
    the (k+1) x (k+1) normal matrix):
        c   = m^T Sigma^-1 m   = the sum of the window's block of Sigma^-1
                                  (m = -1 on the window, 0 elsewhere),
        b   = X^T Sigma^-1 m   = -(column sums of Sigma^-1 X over the window),
        num = m^T Sigma^-1 r0  = -(sum of Sigma^-1 r0 over the window),
              r0 = f - X w_null the residual of the transit-free fit,
        s   = c - b^T (X^T Sigma^-1 X)^-1 b,
        depth = num / s, var = 1 / s (the last diagonal entry of
        (X'^T Sigma^-1 X')^-1), gain = depth^2 / (2 var), which is
        ln L - ln L_null of Eq. linear_search_ll at the GLS weights.
    The transit-free fit w_null is the model's (QR of the whitened X).
    Returns depth, var, dlnl of shape (n_D, n_t0); an empty window (or
    s <= 0) gives NaN.
    """
    from scipy.linalg import lapack

    t0s = np.asarray(t0s, dtype=np.float64)
    Ds = np.asarray(Ds, dtype=np.float64)
    C = model.C
    inv, info = lapack.dpotri(C, lower=1)       # lower triangle of Sigma^-1
    if info != 0:
        raise np.linalg.LinAlgError(f"dpotri failed ({info})")
    yw = model.yw
    if model.k:
        w0, _ = _ols_qr(model.Xw[None], yw[None])
        r0w = yw - model.Xw @ w0[0]
        SX = solve_triangular(C, model.Xw, lower=True, trans="T")    # Sigma^-1 X
        A = model.Xw.T @ model.Xw                                    # X^T Sigma^-1 X
    else:
        r0w = yw
    z0 = solve_triangular(C, r0w, lower=True, trans="T")              # Sigma^-1 r0
    N = model.N
    diag = {}

    def band(d):
        """(Sigma^-1)[a + d, a] for a = 0 .. N-d-1 (from the lower triangle)."""
        if d not in diag:
            diag[d] = np.ascontiguousarray(np.diagonal(inv, offset=-d))
        return diag[d]

    out = {name: np.full((len(Ds), len(t0s)), np.nan) for name in ("depth", "var", "dlnl")}
    for j, D in enumerate(Ds):
        lo, hi = box_windows(model.t, t0s, D)
        L = hi - lo
        for Lv in np.unique(L[L > 0]):
            sel = np.nonzero(L == Lv)[0]
            a0 = lo[sel][:, None]
            win = a0 + np.arange(Lv)[None, :]
            # block sum of Sigma^-1 over the window, diagonal by diagonal:
            # the main diagonal once, every off-diagonal twice (symmetry)
            c = band(0)[win].sum(axis=1)
            for d in range(1, int(Lv)):
                c = c + 2.0 * band(d)[a0 + np.arange(Lv - d)[None, :]].sum(axis=1)
            num = -z0[win].sum(axis=1)
            s = c
            if model.k:
                bx = -SX[win].sum(axis=1)                       # (n_sel, k)
                s = c - np.einsum("bk,bk->b", bx, np.linalg.solve(A, bx.T).T)
            ok = s > 0.0
            i = sel[ok]
            out["depth"][j, i] = num[ok] / s[ok]
            out["var"][j, i] = 1.0 / s[ok]
            out["dlnl"][j, i] = 0.5 * num[ok] * num[ok] / s[ok]
    out["logdet"] = model.logdet
    out["lnL_null"] = model.lnL_null
    return out
