"""Seeded synthetic TESS-shaped light curves and search grids.

This module only draws inputs: time stamps with gaps, quasi-periodic stellar
variability, white noise and injected box dips, plus the (t0, D, P) grids of
the standard workloads.  It holds none of the search arithmetic (no kernel
function, no covariance, no least squares), so the CUDA path and the CPU
oracle can both consume its output without sharing any computation.

The variability is a pair of driven second-order autoregressive sequences with
poles placed at the rotation period and at half of it.  It is a rotation-like
signal of the requested standard deviation; it is not claimed to be an exact
draw from the Gaussian process that the search assumes, and nothing depends
on that.

Workloads (the paper's TESS light curves are not available, so these stand in
for them: 2-minute cadence, ~27-day sectors with a mid-sector gap, rotation
periods from a fraction of a day to days):

* ``single_2048``   N=2048 uniform, P_rot 0.5 d, 5 durations 0.5-2 h, 1000 periods 0.3-1.4 d.
* ``sector_19440``  one sector, 19 440 samples, 1-day mid gap, P_rot 1.2 d,
                    10 durations 20 min-3 h, 20 000 periods 0.2-13.5 d.
* ``sector_19440_16d`` the same sector with 16 durations (mixed precision).
* ``survey_438``    438 light curves, N ~ U[8000, 20000], 1-3 random gaps.
* ``multisector_136080`` seven sectors with 1-day gaps, 20 durations 15 min-4 h,
                    100 000 periods 0.2-50 d.
* ``injection_4000`` the simulated injection-recovery set-up of Sect. 3 (its
                    first comparison): 4000 curves of 4 days at 2 min (N = 2880),
                    white noise 0.1 %, a common transit P = 1.1 d, T0 = 0.2 d,
                    D = 0.04 d, depth 1 %, and SHO variability whose frequency and
                    amplitude follow Eq. relative_params from tau ~ U(0.1, 10),
                    delta ~ U(0.1, 25), with Q ~ U(10, 100); searched with the
                    same SHO kernel, the one duration and 4000 periods 0.3-3 d.
"""
from __future__ import annotations

import dataclasses
import numpy as np
from scipy.signal import lfilter

CADENCE_DAYS = 2.0 / 1440.0
BASE_SEED = 20240206

# term kinds, shared vocabulary with the C ABI (kind codes)
TERM_SHO = 0
TERM_EXP = 1
TERM_ROTATION = 2


@dataclasses.dataclass
class LightCurve:
    t: np.ndarray          # (N,) days, strictly increasing
    y: np.ndarray          # (N,) relative flux
    diag_var: np.ndarray   # (N,) white-noise variance per sample
    terms: list            # [(kind, (p0, p1, p2, p3, p4)), ...]
    X: np.ndarray          # (N, k) design matrix, columns [1, t]
    injected: dict         # {"depth", "duration", "period", "epoch"} or {}


@dataclasses.dataclass
class Workload:
    name: str
    curves: list           # list[LightCurve]
    durations: np.ndarray  # (n_D,) days
    periods: np.ndarray    # (n_P,) days
    seed: int


def _ar2_variability(rng, n_slots, period_days, q, sigma):
    """Driven second-order autoregression with a spectral peak at ``period``."""
    theta = 2.0 * np.pi * CADENCE_DAYS / period_days
    radius = np.exp(-theta / (2.0 * q))
    a1 = 2.0 * radius * np.cos(theta)
    a2 = -radius * radius
    burn = 4000
    e = rng.standard_normal(n_slots + burn)
    x = lfilter([1.0], [1.0, -a1, -a2], e)[burn:]
    sd = x.std()
    return x * (sigma / sd) if sd > 0 else x


def _rotation_signal(rng, n_slots, p_rot, sigma, q0=5.0, frac=0.5):
    """Rotation-like variability: modes at p_rot and p_rot/2, total std sigma."""
    s1 = sigma / np.sqrt(1.0 + frac)
    s2 = sigma * np.sqrt(frac / (1.0 + frac))
    return (_ar2_variability(rng, n_slots, p_rot, 0.5 + q0, s1)
            + _ar2_variability(rng, n_slots, 0.5 * p_rot, 0.5 + q0, s2))


def _inject_box(t, y, depth, duration, period, epoch):
    k0 = np.floor((t[0] - epoch) / period) - 1
    k1 = np.ceil((t[-1] - epoch) / period) + 1
    for k in np.arange(k0, k1 + 1):
        tc = epoch + k * period
        y[np.abs(t - tc) < 0.5 * duration] -= depth
    return y


def make_curve(rng, slots_keep, t_start, p_rot, sigma, sigma_w, q0=5.0,
               inject=None, design=True, n_slots=None):
    """Build one light curve on the 2-min slot grid; keep ``slots_keep``."""
    if n_slots is None:
        n_slots = int(slots_keep[-1]) + 1
    t_all = t_start + np.arange(n_slots) * CADENCE_DAYS
    var = _rotation_signal(rng, n_slots, p_rot, sigma, q0=q0)
    noise = sigma_w * rng.standard_normal(n_slots)
    t = t_all[slots_keep]
    y = 1.0 + var[slots_keep] + noise[slots_keep]
    injected = {}
    if inject is not None:
        depth, duration, period = inject
        # epoch placed on a sample, within the first period
        first = t[t < t[0] + period]
        epoch = float(first[rng.integers(0, len(first))])
        y = _inject_box(t, y, depth, duration, period, epoch)
        injected = dict(depth=depth, duration=duration, period=period, epoch=epoch)
    X = np.stack([np.ones_like(t), t], axis=1) if design else np.zeros((len(t), 0))
    terms = [(TERM_ROTATION, (sigma, p_rot, q0, 0.0, 0.5))]
    return LightCurve(t=t, y=y, diag_var=np.full(len(t), sigma_w ** 2),
                      terms=terms, X=X, injected=injected)


def sector_slots(n_keep=19440, gap_slots=720):
    """Slot indices of one sector: n_keep samples with a centred gap."""
    half = n_keep // 2
    return np.concatenate([np.arange(half),
                           np.arange(half + gap_slots, n_keep + gap_slots)])


def single_2048(seed_offset=0):
    rng = np.random.default_rng(BASE_SEED + 0 + seed_offset)
    lc = make_curve(rng, np.arange(2048), 0.0, 0.5, 1e-2, 1e-3,
                    inject=(2e-3, 1.0 / 24.0, 0.7))
    return Workload("single_2048", [lc], np.linspace(0.5, 2.0, 5) / 24.0,
                    np.linspace(0.3, 1.4, 1000), BASE_SEED + 0)


def sector_19440(n_durations=10, seed_index=1, name="sector_19440"):
    rng = np.random.default_rng(BASE_SEED + seed_index)
    lc = make_curve(rng, sector_slots(), 0.0, 1.2, 2e-2, 2e-3,
                    inject=(1.5e-3, 1.5 / 24.0, 3.1))
    return Workload(name, [lc],
                    np.linspace(20.0 / 1440.0, 3.0 / 24.0, n_durations),
                    np.linspace(0.2, 13.5, 20000), BASE_SEED + seed_index)


def sector_19440_16d():
    return sector_19440(n_durations=16, seed_index=2, name="sector_19440_16d")


def survey_438(n_curves=438, seed_index=3):
    rng = np.random.default_rng(BASE_SEED + seed_index)
    curves = []
    for c in range(n_curves):
        n = int(rng.integers(8000, 20001))
        n_gaps = int(rng.integers(1, 4))
        total = n
        # gaps of 0.2-1.5 d placed at random inside the span
        gaps = []
        for _ in range(n_gaps):
            g = int(rng.uniform(0.2, 1.5) / CADENCE_DAYS)
            gaps.append(g)
        n_slots = n + sum(gaps)
        keep = np.ones(n_slots, dtype=bool)
        for g in gaps:
            s = int(rng.integers(500, n_slots - g - 500))
            keep[s:s + g] = False
        slots = np.nonzero(keep)[0][:total]
        p_rot = float(np.exp(rng.uniform(np.log(0.1), np.log(5.0))))
        sigma = float(np.exp(rng.uniform(np.log(1e-3), np.log(5e-2))))
        sigma_w = float(rng.uniform(1e-3, 5e-3))
        inject = None
        if c % 2 == 0:
            inject = (float(np.exp(rng.uniform(np.log(5e-4), np.log(5e-3)))),
                      float(rng.uniform(0.5, 3.0)) / 24.0,
                      float(rng.uniform(0.5, 10.0)))
        curves.append(make_curve(rng, slots, 0.0, p_rot, sigma, sigma_w,
                                 inject=inject))
    return Workload("survey_438", curves,
                    np.linspace(20.0 / 1440.0, 3.0 / 24.0, 10),
                    np.linspace(0.3, 10.0, 4000), BASE_SEED + seed_index)


def multisector_136080(seed_index=4):
    rng = np.random.default_rng(BASE_SEED + seed_index)
    one = sector_slots()
    span = int(one[-1]) + 1 + 720          # sector slots + 1-day gap
    slots = np.concatenate([one + s * span for s in range(7)])
    lc = make_curve(rng, slots, 0.0, 1.2, 2e-2, 2e-3,
                    inject=(1.5e-3, 1.5 / 24.0, 3.1))
    return Workload("multisector_136080", [lc],
                    np.linspace(15.0 / 1440.0, 4.0 / 24.0, 20),
                    np.linspace(0.2, 50.0, 100000), BASE_SEED + seed_index)


def small_curve(n=300, seed=7, p_rot=0.5, sigma=1e-2, sigma_w=1e-3, gap=None,
                inject=(3e-3, 1.0 / 24.0, 0.31), design=True):
    """A short curve for quick tests (optionally with a gap of ``gap`` slots)."""
    rng = np.random.default_rng(seed)
    if gap is None:
        slots = np.arange(n)
    else:
        half = n // 2
        slots = np.concatenate([np.arange(half), np.arange(half + gap, n + gap)])
    return make_curve(rng, slots, 0.0, p_rot, sigma, sigma_w, inject=inject,
                      design=design)


def injection_4000(n_curves=4000, seed_index=5):
    """Sect. 3's simulated injection-recovery curves (see the module notes).

    Eq. relative_params ties the SHO kernel to the transit: tau = pi/(omega D)
    and delta = 2 sigma / depth, so omega = pi/(tau D) and sigma = delta
    depth / 2.  The variability is the driven AR(2) sequence with its peak at
    the SHO's period 2 pi / omega and quality Q (a stand-in, as elsewhere in
    this module); the search kernel is the SHO (sigma, omega, Q) itself.
    """
    rng = np.random.default_rng(BASE_SEED + seed_index)
    n, depth, duration, period, epoch = 2880, 1e-2, 0.04, 1.1, 0.2
    sigma_w = 1e-3
    t = np.arange(n) * CADENCE_DAYS
    curves = []
    for _ in range(n_curves):
        tau = float(rng.uniform(0.1, 10.0))
        delta = float(rng.uniform(0.1, 25.0))
        q = float(rng.uniform(10.0, 100.0))
        omega = np.pi / (tau * duration)
        sigma = delta * depth / 2.0
        var = _ar2_variability(rng, n, 2.0 * np.pi / omega, q, sigma)
        y = 1.0 + var + sigma_w * rng.standard_normal(n)
        y = _inject_box(t, y, depth, duration, period, epoch)
        curves.append(LightCurve(
            t=t.copy(), y=y, diag_var=np.full(n, sigma_w ** 2),
            terms=[(TERM_SHO, (sigma, omega, q, 0.0, 0.0))],
            X=np.stack([np.ones(n), t], axis=1),
            injected=dict(depth=depth, duration=duration, period=period, epoch=epoch,
                          tau=tau, delta=delta, Q=q)))
    return Workload("injection_4000", curves, np.array([duration]),
                    np.linspace(0.3, 3.0, 4000), BASE_SEED + seed_index)


WORKLOADS = {
    "single_2048": single_2048,
    "sector_19440": sector_19440,
    "sector_19440_16d": sector_19440_16d,
    "survey_438": survey_438,
    "multisector_136080": multisector_136080,
    "injection_4000": injection_4000,
}
