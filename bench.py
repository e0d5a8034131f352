#!/usr/bin/env python
"""Benchmark of the nuance hot path on GB300 (one JSON line on rank 0).

A step is one full pass of the hot path over one light curve of the workload:
nu_gp_factor (covariance factor and null fit), nu_linear_search (every
(t0, D) template) and nu_periodic_search (every trial period), inputs resident
in HBM.  Headline workload: one TESS-sector-shaped light curve, N = 19 440 with
a 1-day mid-sector gap, 10 durations (20 min - 3 h), 20 000 periods
(0.2 - 13.5 d), FP64.  Measured beside it, as keys of the same line:

* mixed_c2:    the same sector in mixed precision (mixed vs FP64 per curve);
* mixed:       the sector with 16 durations in mixed precision;
* multisector: seven sectors (N = 136 080, 20 durations, 100 000 periods),
               FP64 and mixed side by side;
* batch_fp64 / batch_mixed: the 438-curve survey through nu_batch_search;
* cpu_baseline (rank 0, one GPU): the CPU oracle on bounded samples,
               extrapolated, the small light curve's oracle timed in full as
               an anchor, and the mixed path's per-output error against the
               oracle's whole grid of the 16-duration sector.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the CPU oracle (dense FP64 covariance, one GLS per
template, literal Eq. result fold) is timed on the host cores: every step is a
bounded sample of the headline workload (the same sample as cpu_baseline) and
the throughput is extrapolated to a full step.  Multi-GPU (torchrun): every
rank searches its own replica (independent light curves, no data-path
collective; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_06835_gb300 import synth  # noqa: E402

METRIC = "linear-search (t0,D) fits/s + period trials/s, %HBM roofline, mixed vs FP64"
MEASURED_FP64_TFLOPS = 1.197   # DFMA microbenchmark on this machine's GB300 (2 DFMA/clk/SM)
N_SMSP = 152 * 4               # SM sub-partitions (one warp instruction issued per clock each)
# Per launch of the fold (FP64 on the sector, mixed on the 16-duration sector),
# from one-pass ncu captures of the kernels as they stand (the launch lists and
# counters are summarised under profiles/): DRAM bytes read + written, warp
# instructions.
FOLD_NCU = {("sector_19440", "fp64"): {"traffic": 20915456, "inst": 6200356940},
            ("sector_19440_16d", "mixed"): {"traffic": 7206912, "inst": 7679427940}}
FLUSH_BYTES = 512 << 20        # > 129 MB L2
ORACLE_TEMPLATES = 256         # bounded oracle sample per step (both CPU legs)
ORACLE_PERIODS = 8


def measured_peaks():
    """HBM copy bandwidth from the machine's measured peaks, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def linear_search_roofline(lc, Ds, ms, nb=2, k=2):
    """Algorithmic bytes and FP64 flops of one box nu_linear_search with the
    window-start recursion: per sample the factor arrays it reads (t, F, kg,
    1/D, G, z0, Zt), per template the three FP64 outputs; per window start one
    recursion over the longest window (8 + 6 J flops per step: innovation,
    its square, the sums and the gain and transition updates), per template
    the tail s^T G s and the epilogue."""
    J = 2 * nb
    JJ = J * (J + 1) // 2
    n = len(lc.t)
    dt = float(np.median(np.diff(lc.t)))
    lmax = max(int(round(D / dt)) for D in Ds)
    flops = n * lmax * (8 + 6 * J) + n * len(Ds) * (2 * JJ + 2 * J + 20)
    bytes_ = n * 8 * (1 + 4 * nb + J + 1 + JJ + 1 + k) + n * len(Ds) * 24
    hbm, src = measured_peaks()
    gbs = bytes_ / (ms / 1e3) / 1e9
    tfl = flops / (ms / 1e3) / 1e12
    return {"bytes": bytes_, "GB/s": gbs, "hbm_frac": gbs / hbm, "hbm_peak": hbm,
            "hbm_peak_source": src, "fp64_flops": flops, "fp64_tflops": tfl,
            "fp64_pipe_frac": tfl / MEASURED_FP64_TFLOPS,
            "fp64_peak_source": "builder-measured DFMA microbenchmark (1.197 TFLOP/s)"}


def fold_roofline(n_t0, n_D, n_P, ms, visits, value_bytes, kernel, ncu=None, clock_mhz=None):
    """The fold against HBM on its compulsory bytes (the single-event grid read
    once: 3 values of value_bytes per (duration, epoch); 44 bytes of outputs
    per period) and, where an ncu instruction count is at hand, its
    instruction issue rate (the fold is bound by issue and gather latency, not
    by memory bandwidth)."""
    hbm, src = measured_peaks()
    comp = 3 * n_D * n_t0 * value_bytes + 44 * n_P
    gbs = comp / (ms / 1e3) / 1e9
    out = {"kernel": kernel, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
           "frac": gbs / hbm, "traffic": None, "algorithmic_bytes": comp,
           "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
           "timing": "nu_periodic_search stage (the fold kernel and its small prep kernels), "
                     "CUDA events over the timed steps"}
    out["visits"] = visits
    if ncu and ncu.get("traffic"):
        out["traffic"] = ncu["traffic"]
    if ncu and ncu.get("inst") and clock_mhz:
        cyc = ms / 1e3 * clock_mhz * 1e6
        out["issue"] = {"warp_inst_per_launch": ncu["inst"],
                        "frac": ncu["inst"] / (cyc * N_SMSP),
                        "peak": "one warp instruction per clock per sub-partition, "
                                "608 sub-partitions at the sampled SM clock"}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sector_19440")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-multisector", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-refine", action="store_true")
    ap.add_argument("--case", default=None, choices=["fold_small", "batch_small"],
                    help="profiling cases for ncu captures: fold_small = one periodic "
                         "search per precision on the sector grid with 10 000 periods; "
                         "batch_small = two batched searches per precision of 400 "
                         "injection curves")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def fold_visits(t0s, periods, dt, n_D):
    """Exact number of epoch evaluations (per pass) of one periodic search."""
    span = t0s[-1] - t0s[0]
    total = 0
    for P in periods:
        n_phi = int(np.ceil(P / dt))
        phi = np.arange(n_phi) / n_phi
        K = np.floor((span - phi * P) / P).astype(np.int64) + 1
        total += int(K[K > 0].sum())
    return total * n_D


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ our pipeline
class Pipeline:
    def __init__(self, api, torch, lc, Ds, periods, precision, dev):
        self.api, self.torch = api, torch
        f64 = torch.float64
        self.lc = lc
        self.t = torch.as_tensor(lc.t, dtype=f64, device=dev)
        self.y = torch.as_tensor(lc.y, dtype=f64, device=dev)
        self.dv = torch.as_tensor(lc.diag_var, dtype=f64, device=dev)
        self.X = torch.as_tensor(lc.X, dtype=f64, device=dev)
        self.t0s = self.t
        self.periods_np = np.asarray(periods, dtype=np.float64)
        self.periods = torch.as_tensor(periods, dtype=f64, device=dev)
        self.Ds = [float(d) for d in Ds]
        self.terms = lc.terms
        self.precision = precision
        self.dt = float(np.median(np.diff(lc.t)))
        self.n_templates = len(lc.t) * len(Ds)
        self.n_periods = len(periods)

    def step(self, events=None, keep=False):
        api = self.api
        if events:
            events[0].record()
        f = api.nu_gp_factor(self.t, self.dv, self.terms, self.X, self.y)
        if events:
            events[1].record()
        d, v, l = api.nu_linear_search(f, self.t0s, self.Ds, precision=self.precision)
        if events:
            events[2].record()
        res = api.nu_periodic_search(self.t0s, self.Ds, d, v, l, self.periods,
                                     precision=self.precision, phase_step=self.dt)
        if events:
            events[3].record()
        f.free()
        if keep:
            res["grid"] = (d, v, l)
        return res


def time_pipeline(pipe, torch, steps, warmup, flush):
    for _ in range(warmup):
        pipe.step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k + 1)                       # evict L2 between timed steps
        pipe.step(ev[k])
    torch.cuda.synchronize()
    stages = np.array([[ev[k][s].elapsed_time(ev[k][s + 1]) for s in range(3)]
                       for k in range(steps)])
    return stages                                 # (steps, 3) ms


def pipeline_entry(name, pipe, stages, world, ncu=None, clock_mhz=None):
    """The JSON of one single-curve workload measured with time_pipeline."""
    ms = float(stages.sum(axis=1).mean())
    sm = stages.mean(axis=0)
    lc = pipe.lc
    n_D = len(pipe.Ds)
    fp64 = pipe.precision == "fp64"
    visits = fold_visits(lc.t, pipe.periods_np, pipe.dt, n_D)
    return {"workload": name, "precision": pipe.precision, "ms_per_step": ms,
            "value": world * pipe.n_templates / (ms / 1e3), "unit": "(t0,D) fits/s",
            "period_trials_per_s": world * pipe.n_periods / (ms / 1e3),
            "stages_ms": {"factor": float(sm[0]), "linear_search": float(sm[1]),
                          "periodic_search": float(sm[2])},
            "linear_search_fits_per_s": pipe.n_templates / (float(sm[1]) / 1e3),
            "fold_visits_per_s": visits / (float(sm[2]) / 1e3),
            "roofline": fold_roofline(len(lc.t), n_D, pipe.n_periods, float(sm[2]), visits,
                                      8 if fp64 else 4,
                                      "k_fold_screened" if fp64 else "k_fold_slots",
                                      ncu, clock_mhz)}


def run_e2e(pipe, api, torch, lc, steps):
    """Same step through the public API with inputs from pinned host memory,
    outputs read back to the host, copies inside the timed region."""
    f64 = torch.float64
    host = {k: torch.as_tensor(np.ascontiguousarray(v), dtype=f64).pin_memory()
            for k, v in (("t", lc.t), ("y", lc.y), ("dv", lc.diag_var), ("X", lc.X),
                         ("P", pipe.periods_np))}
    dev = {k: torch.empty_like(v, device="cuda") for k, v in host.items()}
    nP = pipe.n_periods
    out_host = torch.empty((5, nP), dtype=f64).pin_memory()
    idx_host = torch.empty(nP, dtype=torch.int32).pin_memory()
    bi = sum(v.numel() * v.element_size() for v in host.values())
    bo = out_host.numel() * 8 + idx_host.numel() * 4

    def one():
        for k in host:
            dev[k].copy_(host[k], non_blocking=True)
        f = api.nu_gp_factor(dev["t"], dev["dv"], pipe.terms, dev["X"], dev["y"])
        d, v, l = api.nu_linear_search(f, dev["t"], pipe.Ds, precision=pipe.precision)
        r = api.nu_periodic_search(dev["t"], pipe.Ds, d, v, l, dev["P"],
                                   precision=pipe.precision, phase_step=pipe.dt)
        out_host.copy_(torch.stack([r["Q"], r["T0"], r["depth"], r["sigma"], r["lnP"]]),
                       non_blocking=True)
        idx_host.copy_(r["D_idx"], non_blocking=True)
        f.free()

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return ms, bi, bo


# --------------------------------------------- exact fit of the top periods
def run_refine(pipe, api, torch, n_top=64, reps=5):
    """nu_periodic_refine on the search's best n_top periods: the exact fit of
    a periodic transit column at full covariance.  Timed alone (CUDA events);
    also reports Eq. result's Q against the exact SNR at the best period."""
    res = pipe.step()
    f = api.nu_gp_factor(pipe.t, pipe.dv, pipe.terms, pipe.X, pipe.y)
    Q = torch.nan_to_num(res["Q"], nan=-1.0)
    top = torch.argsort(Q, descending=True)[:n_top]
    P = pipe.periods[top].contiguous()
    T0 = res["T0"][top].contiguous()
    J = res["D_idx"][top].contiguous()
    r = api.nu_periodic_refine(f, P, T0, J, pipe.Ds)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        api.nu_periodic_refine(f, P, T0, J, pipe.Ds)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    q, snr = float(Q[top[0]]), float(r["snr"][0])
    f.free()
    return {"n_candidates": int(top.numel()), "ms": ms,
            "candidates_per_s": top.numel() / (ms / 1e3),
            "best_period": float(P[0]), "Q_eq_result": q, "snr_exact": snr,
            "rel_diff": abs(snr - q) / q if q > 0 else None}


# ------------------------------------------------------------ batch (C4)
def recovery(w, r):
    """Sect. 3's detection rule on the batch result, for workloads whose
    curves all carry the same injected period p: a curve counts as recovered
    when its best period is within 0.01 d of p, 2p or p/2 and its Q >= 6."""
    ps = {lc.injected.get("period") for lc in w.curves}
    if len(ps) != 1 or None in ps:
        return {}
    p = ps.pop()
    Q = r["Q"].double().cpu().numpy()
    Q = np.where(np.isfinite(Q), Q, -np.inf)
    best = np.argmax(Q, axis=1)
    pb = w.periods[best]
    qb = Q[np.arange(len(best)), best]
    near = np.min(np.abs(pb[:, None] - np.array([p, 2 * p, p / 2])[None, :]), axis=1) < 0.01
    hit = near & (qb >= 6.0)
    return {"recovered_fraction": float(hit.mean()), "recovered": int(hit.sum()),
            "curves": int(len(hit))}


def run_batch(api, torch, w, precision, steps, warmup, flush):
    """nu_batch_search over all curves of a survey workload; one step = one
    batched call (factor, linear search and fold of every curve)."""
    items = [(torch.as_tensor(lc.t, device="cuda"), torch.as_tensor(lc.y, device="cuda"),
              torch.as_tensor(lc.diag_var, device="cuda"), lc.terms) for lc in w.curves]
    periods = torch.as_tensor(w.periods, dtype=torch.float64, device="cuda")
    dt = synth.CADENCE_DAYS
    for _ in range(warmup):
        api.nu_batch_search(items, w.durations, periods, k=2, precision=precision,
                            phase_step=dt)
    torch.cuda.synchronize()
    times = []
    for k in range(steps):
        flush.fill_(k + 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = api.nu_batch_search(items, w.durations, periods, k=2, precision=precision,
                                phase_step=dt)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    n_samples = sum(len(lc.t) for lc in w.curves)
    n_templates = n_samples * len(w.durations)
    ms = float(np.mean(times))
    out_rec = recovery(w, r)
    hbm, src = measured_peaks()
    comp = n_samples * 8 * 3 + 44 * len(w.periods) * len(w.curves)
    return {**out_rec, "workload": f"{w.name}: {len(w.curves)} curves, {n_samples} samples, "
                                   f"{len(w.durations)} durations, {len(w.periods)} periods",
            "precision": precision, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "value": n_templates / (ms / 1e3), "unit": "(t0,D) fits/s",
            "period_trials_per_s": len(w.curves) * len(w.periods) / (ms / 1e3),
            "failed_curves": int(sum(1 for s_ in r["status"] if s_ != 0)),
            "roofline": {"bound": "hbm", "unit": "GB/s", "algorithmic_bytes": comp,
                         "achieved": comp / (ms / 1e3) / 1e9, "peak": hbm,
                         "frac": comp / (ms / 1e3) / 1e9 / hbm, "peak_source": src,
                         "note": "compulsory bytes of the whole batched call: the light "
                                 "curves (t, y, variance) once and 44 B of outputs per "
                                 "(curve, period); one CUDA graph, timed with CUDA events"}}


# ---------------------------------------------------------------- ranks
def max_over_ranks(ms, torch, device):
    """Slowest rank's time (every rank gets it); identity without a group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(ms)
    tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def weak_scaling_value(units_per_rank, world, ms):
    """Whole-job throughput: every rank processed its own units in <= ms."""
    return world * units_per_rank / (ms / 1e3)


# ---------------------------------------------------------------- oracle
def oracle_sample(lc, Ds, periods, model, t_setup, n_templates=ORACLE_TEMPLATES,
                  n_periods=ORACLE_PERIODS, seed=0):
    """Time the oracle on a bounded sample of one step (random templates, random
    periods of the fold on a grid of the step's shape) and extrapolate to the
    full step.  The dense factor, built once, is counted in every step."""
    from oracle import linear, periodic
    rng = np.random.default_rng(seed)
    n = len(lc.t)
    w0 = time.perf_counter()
    pairs = [(int(rng.integers(0, len(Ds))), int(rng.integers(0, n)))
             for _ in range(n_templates)]
    t0 = time.perf_counter()
    linear.sampled_linear_search(model, lc.t, Ds, pairs)
    t_lin = (time.perf_counter() - t0) / n_templates
    # fold on a synthetic grid of the right shape (values do not change the work)
    g = dict(depth=rng.normal(0, 1e-3, (len(Ds), n)), var=rng.uniform(1e-8, 4e-8, (len(Ds), n)),
             dlnl=rng.uniform(0, 5, (len(Ds), n)))
    sel = rng.choice(len(periods), size=n_periods, replace=False)
    dt = float(np.median(np.diff(lc.t)))
    t0 = time.perf_counter()
    periodic.periodic_search(lc.t, g["depth"], g["var"], g["dlnl"], np.asarray(periods)[sel], dt)
    t_per = (time.perf_counter() - t0) / n_periods
    total = t_setup + t_lin * n * len(Ds) + t_per * len(periods)
    return dict(t_template=t_lin, t_period=t_per, total_s=total,
                wall_s=time.perf_counter() - w0,
                sample=f"dense Sigma factor once ({t_setup:.1f} s, counted in every step), "
                       f"{n_templates} random templates, {n_periods} random periods; "
                       f"extrapolated to {n * len(Ds)} templates + {len(periods)} periods")


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_legs(lc, w, n_templates, gpu_mixed16):
    """The oracle on the host cores (bench.py's CPU baseline leg): the headline
    workload on a bounded sample, extrapolated; the 2048-sample light curve in
    full (the anchor of the extrapolations); the seven-sector curve through the
    sequential celerite reference (bounded sample, extrapolated); the survey
    from its shortest curve (bounded sample, extrapolated); and the mixed
    path's per-output error against the oracle's whole grid of the 16-duration
    sector (gpu_mixed16: the GPU's mixed linear search and fold of that
    workload)."""
    from oracle import linear, periodic, semisep
    out = {}
    t0 = time.perf_counter()
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    t_setup = time.perf_counter() - t0
    s = oracle_sample(lc, w.durations, w.periods, model, t_setup)
    out["cpu_baseline"] = {"value": n_templates / s["total_s"], "unit": "(t0,D) fits/s",
                           "cores": blas_threads(), "kind": "oracle", "extrapolated": True,
                           "sample": s["sample"], "wall_s": s["wall_s"] + t_setup,
                           "period_trials_per_s": len(w.periods) / s["total_s"]}
    del model
    # anchor: the 2048-sample light curve's oracle in full (10 240 templates,
    # 1000 periods), against the same extrapolation from a bounded sample
    w1 = synth.single_2048()
    l1 = w1.curves[0]
    t0 = time.perf_counter()
    m1 = linear.DenseModel(l1.t, l1.y, l1.diag_var, l1.terms, l1.X)
    ts1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    o1 = linear.linear_search(l1.t, l1.y, l1.diag_var, l1.terms, l1.X, l1.t, w1.durations,
                              model=m1)
    tl1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    periodic.periodic_search(l1.t, o1["depth"], o1["var"], o1["dlnl"], w1.periods,
                             periodic.median_spacing(l1.t))
    tp1 = time.perf_counter() - t0
    full = ts1 + tl1 + tp1
    s1 = oracle_sample(l1, w1.durations, w1.periods, m1, ts1, seed=1)
    out["cpu_anchor_single_2048"] = {
        "full_s": full, "value": len(l1.t) * len(w1.durations) / full,
        "unit": "(t0,D) fits/s", "period_trials_per_s": len(w1.periods) / full,
        "extrapolated": False, "sample_extrapolation_s": s1["total_s"],
        "extrapolation_ratio": s1["total_s"] / full}
    # seven sectors: the celerite reference (the dense Sigma would need 148 GB)
    w5 = synth.multisector_136080()
    l5 = w5.curves[0]
    rng = np.random.default_rng(5)
    t0 = time.perf_counter()
    ss = semisep.Semisep(l5.t, l5.diag_var, l5.terms)
    ts5 = time.perf_counter() - t0
    pairs = [(int(rng.integers(0, len(w5.durations))), int(rng.integers(0, len(l5.t))))
             for _ in range(16)]
    t0 = time.perf_counter()
    semisep.sampled_linear_search(l5.t, l5.y, l5.diag_var, l5.terms, l5.X, w5.durations, pairs,
                                  model=ss)
    tt5 = (time.perf_counter() - t0) / len(pairs)
    g5 = dict(depth=rng.normal(0, 5e-4, (len(w5.durations), len(l5.t))),
              var=rng.uniform(2e-8, 9e-8, (len(w5.durations), len(l5.t))),
              dlnl=rng.uniform(0, 6, (len(w5.durations), len(l5.t))))
    t0 = time.perf_counter()
    periodic.periodic_search(l5.t, g5["depth"], g5["var"], g5["dlnl"],
                             w5.periods[rng.choice(len(w5.periods), 3, replace=False)],
                             periodic.median_spacing(l5.t))
    tpp5 = (time.perf_counter() - t0) / 3
    tot5 = ts5 + tt5 * len(l5.t) * len(w5.durations) + tpp5 * len(w5.periods)
    out["cpu_multisector"] = {
        "value": len(l5.t) * len(w5.durations) / tot5, "unit": "(t0,D) fits/s",
        "period_trials_per_s": len(w5.periods) / tot5, "kind": "celerite reference "
        "(oracle/semisep.py, the stand-in where the dense oracle does not fit)",
        "extrapolated": True, "sample": f"factor once ({ts5:.1f} s), 16 templates, 3 periods"}
    # survey (438 curves in one batched call on the GPU): the oracle on its
    # shortest curve (dense factor and a bounded sample), extrapolated to every
    # curve: the factor by (n / n0)^3, templates by count, folds by span
    w4 = synth.survey_438()
    lens = np.array([len(c.t) for c in w4.curves])
    l4 = w4.curves[int(np.argmin(lens))]
    t0 = time.perf_counter()
    m4 = linear.DenseModel(l4.t, l4.y, l4.diag_var, l4.terms, l4.X)
    ts4 = time.perf_counter() - t0
    s4 = oracle_sample(l4, w4.durations, w4.periods, m4, ts4, n_templates=64, n_periods=4,
                       seed=4)
    del m4
    n0, span0 = len(l4.t), float(l4.t[-1] - l4.t[0])
    tot4 = sum(ts4 * (len(c.t) / n0) ** 3 + s4["t_template"] * len(c.t) * len(w4.durations) +
               s4["t_period"] * len(w4.periods) * float(c.t[-1] - c.t[0]) / span0
               for c in w4.curves)
    out["cpu_survey"] = {
        "value": float(lens.sum()) * len(w4.durations) / tot4, "unit": "(t0,D) fits/s",
        "period_trials_per_s": len(w4.curves) * len(w4.periods) / tot4,
        "cores": blas_threads(), "kind": "oracle", "extrapolated": True,
        "sample": f"the shortest of {len(w4.curves)} curves (N={n0}): dense Sigma factor "
                  f"({ts4:.1f} s), 64 random templates, 4 random periods; extrapolated to "
                  f"every curve (factor x (N/N0)^3, templates by count, folds by span)",
        "wall_s": ts4 + s4["wall_s"]}
    # mixed precision: per-output error against the FP64 oracle's whole grid
    if gpu_mixed16 is not None:
        out["mixed_error"] = mixed_error(gpu_mixed16)
    return out


def mixed_error(gpu):
    """Largest error of every output of the mixed path on the 16-duration
    sector against the FP64 oracle: the linear search on every template (depth
    relative to max(|depth|, sigma), variance relative, gain relative to
    max(gain, 1)) and the fold on sampled periods (ln P relative to
    max(1, |ln P|), depth and sigma as for the linear search, Q absolute),
    compared at the GPU's argmax cell."""
    from oracle import linear, periodic
    w = synth.sector_19440_16d()
    lc = w.curves[0]
    t0 = time.perf_counter()
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    o = linear.box_grid(model, lc.t, w.durations)
    d, v, l = (np.asarray(a, dtype=np.float64) for a in gpu["grid"])
    ok = ~(np.isnan(o["depth"]) | np.isnan(d))
    so = np.sqrt(o["var"][ok])
    e_lin = {"depth": float(np.max(np.abs(d[ok] - o["depth"][ok]) /
                                   np.maximum(np.abs(o["depth"][ok]), so))),
             "var": float(np.max(np.abs(v[ok] - o["var"][ok]) / o["var"][ok])),
             "dlnl": float(np.max(np.abs(l[ok] - o["dlnl"][ok]) /
                                  np.maximum(o["dlnl"][ok], 1.0))),
             "templates": int(ok.sum()),
             "nan_pattern_equal": bool(np.array_equal(np.isnan(o["depth"]), np.isnan(d)))}
    rng = np.random.default_rng(9)
    q = np.where(np.isfinite(gpu["Q"]), gpu["Q"], -np.inf)
    sel = np.unique(np.concatenate([rng.integers(0, len(w.periods), 40),
                                    np.argsort(-q, kind="stable")[:8]]))
    dt = periodic.median_spacing(lc.t)
    e = dict(lnP=0.0, depth=0.0, sigma=0.0, Q_abs=0.0)
    for p in sel:
        P = w.periods[p]
        f = periodic.fold_period(lc.t, o["depth"], o["var"], o["dlnl"], P, dt)
        dg = int(gpu["D_idx"][p])
        if dg < 0:
            continue
        n_phi = int(np.ceil(P / dt))
        jg = int(np.rint((gpu["T0"][p] - lc.t[0]) / P * n_phi))
        lo, do_, so_ = f["lnP"][dg, jg], f["depth"][dg, jg], f["sigma"][dg, jg]
        best = np.nanmax(np.where(np.isfinite(f["lnP"]), f["lnP"], -np.inf))
        e["lnP"] = max(e["lnP"], abs(gpu["lnP"][p] - best) / max(1.0, abs(best)))
        e["depth"] = max(e["depth"], abs(gpu["depth"][p] - do_) / max(abs(do_), so_))
        e["sigma"] = max(e["sigma"], abs(gpu["sigma"][p] - so_) / so_)
        e["Q_abs"] = max(e["Q_abs"], abs(gpu["Q"][p] - do_ / so_))
    return {"workload": "sector_19440_16d", "linear_search": e_lin,
            "fold": {**e, "periods": int(len(sel))},
            "bounds": {"depth": 1e-4, "Q_abs": 1e-3}, "oracle_s": time.perf_counter() - t0}


# ---------------------------------------------------------------- reference arm
def run_reference(args, w, config):
    """The CPU oracle timed as the reference implementation: every step a
    bounded sample of the headline workload (the same sample size as
    cpu_baseline), extrapolated to a full step."""
    from oracle import linear
    lc = w.curves[0]
    n_templates = len(lc.t) * len(w.durations)
    t0 = time.perf_counter()
    model = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    t_setup = time.perf_counter() - t0
    for k in range(args.warmup):
        oracle_sample(lc, w.durations, w.periods, model, t_setup, seed=1000 + k)
    walls, totals = [], []
    w0 = time.perf_counter()
    for k in range(args.steps):
        r = oracle_sample(lc, w.durations, w.periods, model, t_setup, seed=k + 1)
        walls.append(r["wall_s"])
        totals.append(r["total_s"])
    wall = time.perf_counter() - w0
    tot = statistics.median(totals)
    val = n_templates / tot
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "(t0,D) fits/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(walls) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config, "period_trials_per_s": len(w.periods) / tot,
            "extrapolated": True, "full_step_s_extrapolated": tot,
            "wall_s_timed": wall, "setup_s": t_setup,
            "cpu_baseline": {"value": val, "unit": "(t0,D) fits/s", "cores": blas_threads(),
                             "kind": "oracle", "extrapolated": True,
                             "sample": r["sample"] + "; ms_per_step is the wall time of "
                                                    "one sample step"},
            "e2e": {"value": val, "unit": "(t0,D) fits/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- main
def profile_case(args):
    """Small cases for ncu: the sector light curve (19 440 epochs with the
    mid-sector gap, 10 durations) through nu_gp_factor and nu_linear_search,
    then one nu_periodic_search per precision over 10 000 of its 20 000
    periods (every 2nd, 0.2-13.5 d: enough periods for the folds' launch shapes
    of the full grid)."""
    import torch
    from paper_2402_06835_gb300 import api
    w = synth.sector_19440()
    lc = w.curves[0]
    cu = lambda a: torch.as_tensor(a, device="cuda")
    t = cu(lc.t)
    f = api.nu_gp_factor(t, cu(lc.diag_var), lc.terms, cu(lc.X), cu(lc.y))
    per = cu(np.ascontiguousarray(w.periods[::2]))
    for prec in ("mixed", "fp64"):
        d, v, l = api.nu_linear_search(f, t, w.durations, precision=prec)
        r = api.nu_periodic_search(t, w.durations, d, v, l, per, precision=prec)
        torch.cuda.synchronize()
        print(prec, float(r["Q"].max()))


def profile_batch_case(args):
    """Small batched case for ncu: 400 curves of the injection workload (2880
    samples, 1 duration, 4000 periods), nu_batch_search twice per precision
    (mixed first, then FP64).  The first call of each precision tunes the
    launch shapes; the second runs the chosen ones."""
    import torch
    from paper_2402_06835_gb300 import api
    w = synth.injection_4000(n_curves=400)
    cu = lambda a: torch.as_tensor(a, device="cuda")
    items = [(cu(lc.t), cu(lc.y), cu(lc.diag_var), lc.terms) for lc in w.curves]
    per = cu(w.periods)
    for prec in ("mixed", "fp64"):
        for _ in range(2):
            r = api.nu_batch_search(items, w.durations, per, k=2, precision=prec,
                                    phase_step=synth.CADENCE_DAYS)
        torch.cuda.synchronize()
        print(prec, float(r["Q"].max()))


def main():
    args = parse()
    if args.case == "fold_small":
        profile_case(args)
        return
    if args.case == "batch_small":
        profile_batch_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = synth.WORKLOADS[args.workload]()
    lc = w.curves[0]
    n_templates = len(lc.t) * len(w.durations)
    config = {"workload": f"{args.workload}: N={len(lc.t)} (2-min cadence, gaps), "
                          f"{len(w.durations)} durations, {len(w.periods)} periods, "
                          f"t0 = every sample, X=[1,t], rotation GP (2 SHO, J=4)",
              "n_templates": n_templates, "n_periods": len(w.periods),
              "precision": args.precision, "l2": "flushed (512 MB write) between timed steps"}

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, w, config)))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2402_06835_gb300 import api

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if len(w.curves) > 1:
        # survey workload: the batched call is the step
        b = run_batch(api, torch, w, args.precision, args.steps, args.warmup, flush)
        ms = max_over_ranks(b["ms_per_step"], torch, dev)
        nt = sum(len(lc.t) for lc in w.curves) * len(w.durations)
        out = {"metric": METRIC, "value": weak_scaling_value(nt, world, ms),
               "unit": "(t0,D) fits/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
               "data": "synthetic", "config": {"workload": b["workload"],
                                               "precision": args.precision,
                                               "l2": "flushed (512 MB write) between timed steps"},
               "period_trials_per_s": world * b["period_trials_per_s"], "batch": b}
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    pipe = Pipeline(api, torch, lc, w.durations, w.periods, args.precision, dev)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    # warm up outside the sampler, then time
    for _ in range(args.warmup):
        pipe.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    n0 = api.launch_count()
    sampler = ClockSampler(gpu_id)
    time.sleep(0.4)
    t_wall0 = time.perf_counter()
    stages = time_pipeline(pipe, torch, args.steps, 0, flush)
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    launches = api.launch_count() - n0
    ms = max_over_ranks(float(stages.sum(axis=1).mean()), torch, dev)
    head = pipeline_entry(args.workload, pipe, stages, world,
                          FOLD_NCU.get((args.workload, args.precision)),
                          clocks["sm_mhz"] if clocks else None)
    out = {"metric": METRIC, "value": weak_scaling_value(n_templates, world, ms),
           "unit": "(t0,D) fits/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
           "config": config, "period_trials_per_s": world * len(w.periods) / (ms / 1e3),
           "stages_ms": head["stages_ms"],
           "linear_search_fits_per_s": head["linear_search_fits_per_s"],
           "linear_search_roofline": linear_search_roofline(lc, w.durations,
                                                            head["stages_ms"]["linear_search"]),
           "fold_visits_per_s": head["fold_visits_per_s"],
           "gpu_launches": int(launches), "wall_s_timed": t_wall, "clocks": clocks,
           "roofline": head["roofline"]}

    if not args.no_e2e:
        try:
            e2e_ms, bi, bo = run_e2e(pipe, api, torch, lc, max(1, args.steps))
            out["e2e"] = {"value": world * n_templates / (e2e_ms / 1e3), "unit": "(t0,D) fits/s",
                          "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                          "ms_per_step": e2e_ms}
        except Exception as exc:      # report, do not hide
            out["e2e"] = {"error": repr(exc)}

    extras = world == 1 and args.precision == "fp64"
    if not args.no_refine and extras:
        try:
            out["refine_top64"] = run_refine(pipe, api, torch)
        except Exception as exc:
            out["refine_top64"] = {"error": repr(exc)}

    gpu_mixed16 = None
    if not args.no_mixed and extras:
        for key, wname in (("mixed_c2", "sector_19440"), ("mixed", "sector_19440_16d")):
            try:
                wm = synth.WORKLOADS[wname]()
                pm = Pipeline(api, torch, wm.curves[0], wm.durations, wm.periods, "mixed", dev)
                sm = time_pipeline(pm, torch, args.steps, args.warmup, flush)
                out[key] = pipeline_entry(wname, pm, sm, world)
                if key == "mixed":
                    r = pm.step(keep=True)
                    torch.cuda.synchronize()
                    gpu_mixed16 = {k: v.double().cpu().numpy() for k, v in r.items()
                                   if k != "grid"}
                    gpu_mixed16["grid"] = [a.double().cpu().numpy() for a in r["grid"]]
            except Exception as exc:
                out[key] = {"error": repr(exc)}

    if not args.no_multisector and extras:
        # seven sectors, FP64 and mixed side by side (about a second per step:
        # at most 5 timed steps after 2 warm-ups)
        w5 = synth.multisector_136080()
        ms_steps, ms_warm = min(args.steps, 5), min(args.warmup, 2)
        entry = {"workload": "multisector_136080: N=136080 (7 sectors with 1-day gaps), "
                             "20 durations, 100000 periods",
                 "steps": ms_steps, "warmup": ms_warm}
        for prec in ("fp64", "mixed"):
            try:
                p5 = Pipeline(api, torch, w5.curves[0], w5.durations, w5.periods, prec, dev)
                s5 = time_pipeline(p5, torch, ms_steps, ms_warm, flush)
                entry[prec] = pipeline_entry("multisector_136080", p5, s5, world)
                del p5
            except Exception as exc:
                entry[prec] = {"error": repr(exc)}
        out["multisector"] = entry

    if not args.no_batch and extras:
        # the survey in one batched call, mixed precision and FP64 side by side,
        # with the headline's warm-up and step counts
        survey = synth.survey_438()
        for key, prec in (("batch_mixed", "mixed"), ("batch_fp64", "fp64")):
            try:
                out[key] = run_batch(api, torch, survey, prec, args.steps, args.warmup, flush)
            except Exception as exc:
                out[key] = {"error": repr(exc)}

    if world > 1:
        torch.distributed.barrier()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            legs = cpu_legs(lc, w, n_templates, gpu_mixed16)
            out.update(legs)
            if "cpu_multisector" in legs and isinstance(out.get("multisector"), dict):
                out["multisector"]["cpu_baseline"] = legs.pop("cpu_multisector")
                out.pop("cpu_multisector", None)
            if "cpu_survey" in legs:
                for key in ("batch_mixed", "batch_fp64"):
                    if isinstance(out.get(key), dict) and "error" not in out[key]:
                        out[key]["cpu_baseline"] = legs["cpu_survey"]
                out.pop("cpu_survey", None)
        except Exception as exc:
            out["cpu_baseline"] = {"error": repr(exc)}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
