"""Thin Python binding of the C ABI in include/nuance.h (marshalling only).

Every function here checks shapes and dtypes, passes device pointers and the
current CUDA stream to the library and returns torch tensors that the library
filled.  All arithmetic of the search runs in the CUDA library; there is no
CPU path.  Importing this module loads ``_build/libnuance_gb300.so`` and
raises ImportError if it has not been built (``python -m
paper_2402_06835_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

NU_OK, NU_EINVAL, NU_ENOTPD, NU_ECUDA, NU_ENOMEM, NU_ETIMEOUT = range(6)
NU_FP64, NU_MIXED = 0, 1
NU_BOX, NU_TRAPEZOID, NU_LIMB_QUAD = 0, 1, 2
NU_TERM_SHO, NU_TERM_EXP, NU_TERM_ROTATION = 0, 1, 2

_STATUS_NAMES = {0: "NU_OK", 1: "NU_EINVAL", 2: "NU_ENOTPD", 3: "NU_ECUDA",
                 4: "NU_ENOMEM", 5: "NU_ETIMEOUT"}
_PREC = {"fp64": NU_FP64, "mixed": NU_MIXED}
_TMPL = {"box": NU_BOX, "trapezoid": NU_TRAPEZOID, "limb_quad": NU_LIMB_QUAD}


def _tmpl_params(template, ingress_frac, ld):
    """Host array of the template's parameters (see nu_template)."""
    if template not in _TMPL:
        raise ValueError(f"unknown template {template!r}")
    vals = {"box": (0.0, 0.0), "trapezoid": (float(ingress_frac), 0.0),
            "limb_quad": (float(ld[0]), float(ld[1]))}[template]
    return (ctypes.c_double * 2)(*vals)


class NuanceError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")


class nu_term(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 5)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library {path} not built; run `python -m "
            "paper_2402_06835_gb300.build` (needs nvcc for sm_103a)")
    lib = ctypes.CDLL(path)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.nu_gp_factor.argtypes = [P, P, I64, ctypes.POINTER(nu_term), I, P, I, P, P,
                                 ctypes.POINTER(P)]
    lib.nu_factor_info.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D),
                                   ctypes.POINTER(I64)]
    lib.nu_factor_size.argtypes = [P, ctypes.POINTER(I)]
    lib.nu_factor_size.restype = I64
    lib.nu_factor_free.argtypes = [P]
    lib.nu_factor_free.restype = None
    lib.nu_linear_search.argtypes = [P, P, I64, P, I, I, P, I, P, P, P, P]
    lib.nu_periodic_search.argtypes = [P, I64, P, I, P, P, P, I, P, I64, D, D, P,
                                       P, P, P, P, P, P]
    lib.nu_mask_transits.argtypes = [P, I64, I, P, P, P, I, D, D, D, P]
    lib.nu_mask_transits.restype = I
    lib.nu_periodic_refine.argtypes = [P, P, P, P, I64, P, I, I, P, P, P, P, P, P]
    lib.nu_periodic_refine.restype = I
    lib.nu_rotation_alias_filter.argtypes = [P, I64, D, D, I, P, P, P]
    lib.nu_rotation_alias_filter.restype = I
    lib.nu_periodic_search_noalloc.argtypes = lib.nu_periodic_search.argtypes
    lib.nu_periodic_search_noalloc.restype = I
    lib.nu_periodic_search_noalloc_limit.restype = ctypes.c_uint64
    lib.nu_batch_search.argtypes = [I, P, P, P, P, ctypes.POINTER(nu_term), P, I, P, I,
                                    P, I64, D, I, P, P, P, P, P, P, P, P]
    lib.nu_batch_search.restype = I
    lib.nu_last_error.restype = ctypes.c_char_p
    lib.nu_version.restype = ctypes.c_char_p
    lib.nu_launch_count.restype = ctypes.c_uint64
    for name in ("nu_gp_factor", "nu_factor_info", "nu_linear_search",
                 "nu_periodic_search", "nu_batch_search"):
        getattr(lib, name).restype = I
    return lib


LIB = _load()


def _check(status, what):
    if status != NU_OK:
        raise NuanceError(status, f"{what}: {LIB.nu_last_error().decode()}")


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(x, name, dtype=torch.float64):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype} (got {x.dtype})")
    return x.contiguous()


def _p(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else ctypes.c_void_p(0)


def make_terms(terms):
    """[(kind, params), ...] -> ctypes array of nu_term."""
    arr = (nu_term * max(1, len(terms)))()
    for i, (kind, params) in enumerate(terms):
        arr[i].kind = int(kind)
        vals = list(params) + [0.0] * (5 - len(params))
        for j in range(5):
            arr[i].p[j] = float(vals[j])
    return arr


class Factor:
    """Owner of a nu_factor handle (library device memory)."""

    def __init__(self, handle, n, k, keep, stream):
        self._h = handle
        self.n = n
        self.k = k
        self._keep = keep        # caller tensors read asynchronously
        self.stream = stream

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("factor already freed")
        return self._h

    def info(self):
        """Synchronising read of (status, logdet, lnL_null, first_bad)."""
        ld, ln, fb = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        st = LIB.nu_factor_info(self.handle, ctypes.byref(ld), ctypes.byref(ln),
                                ctypes.byref(fb))
        return dict(status=st, logdet=ld.value, lnL_null=ln.value,
                    first_bad=fb.value,
                    message=LIB.nu_last_error().decode() if st else "")

    def free(self):
        if self._h is not None:
            LIB.nu_factor_free(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def nu_gp_factor(t, diag_var, terms, X, y, stream=None):
    """Factor Sigma and prepare the search vectors (see nu_gp_factor in the header).

    t, diag_var, y: (N,) float64 CUDA tensors; X: (N, k) float64 or None.
    """
    t = _dev(t, "t")
    diag_var = _dev(diag_var, "diag_var")
    y = _dev(y, "y")
    n = t.numel()
    if diag_var.numel() != n or y.numel() != n:
        raise ValueError("t, diag_var and y must have the same length")
    if X is None or X.numel() == 0:
        k, Xc = 0, None
    else:
        X = _dev(X, "X")
        if X.dim() != 2 or X.shape[0] != n:
            raise ValueError("X must be (N, k)")
        k = X.shape[1]
        Xc = X.t().contiguous()                 # column-major (k, N)
    tm = make_terms(terms)
    h = ctypes.c_void_p()
    sp = _stream_ptr(stream)
    st = LIB.nu_gp_factor(_p(t), _p(diag_var), n, tm, len(terms), _p(Xc), k, _p(y),
                          sp, ctypes.byref(h))
    _check(st, "nu_gp_factor")
    return Factor(h, n, k, (t, diag_var, y, Xc), stream)


def nu_factor_info(factor):
    return factor.info()


def nu_linear_search(factor, t0s, Ds, template="box", ingress_frac=0.1,
                     precision="fp64", stream=None, out=None, ld=(0.4, 0.25)):
    """Linear search (Sect. 2.2).  Returns (depth, var, dlnl), each (n_D, n_t0)."""
    t0s = _dev(t0s, "t0s")
    Ds = [float(d) for d in (Ds.tolist() if hasattr(Ds, "tolist") else Ds)]
    n_D, n_t0 = len(Ds), t0s.numel()
    prec = _PREC[precision]
    dt = torch.float64 if prec == NU_FP64 else torch.float32
    if out is None:
        out = tuple(torch.empty((n_D, n_t0), dtype=dt, device=t0s.device)
                    for _ in range(3))
    for o in out:
        if o.dtype != dt or o.numel() != n_D * n_t0 or not o.is_contiguous():
            raise ValueError("output tensors must be contiguous (n_D, n_t0) of the "
                             "precision's dtype")
    Ds_arr = (ctypes.c_double * n_D)(*Ds)
    st = LIB.nu_linear_search(factor.handle, _p(t0s), n_t0, Ds_arr, n_D,
                              _TMPL[template], _tmpl_params(template, ingress_frac, ld), prec,
                              _stream_ptr(stream), _p(out[0]), _p(out[1]), _p(out[2]))
    _check(st, "nu_linear_search")
    return out


def nu_periodic_search(t0s, Ds, depth, var, dlnl, periods, precision="fp64",
                       phase_step=0.0, gap_factor=1.5, stream=None, _entry=None):
    """Periodic search (Sect. 2.3-2.4).  Returns a dict of (n_P,) tensors."""
    t0s = _dev(t0s, "t0s")
    periods = _dev(periods, "periods")
    prec = _PREC[precision]
    dt = torch.float64 if prec == NU_FP64 else torch.float32
    depth, var, dlnl = (_dev(a, nm, dt) for a, nm in
                        ((depth, "depth"), (var, "var"), (dlnl, "dlnl")))
    n_D = depth.shape[0] if depth.dim() == 2 else len(Ds)
    n_P = periods.numel()
    dev = t0s.device
    res = {name: torch.empty(n_P, dtype=torch.float64, device=dev)
           for name in ("Q", "T0", "depth", "sigma", "lnP")}
    res["D_idx"] = torch.empty(n_P, dtype=torch.int32, device=dev)
    Ds_l = [float(d) for d in (Ds.tolist() if hasattr(Ds, "tolist") else Ds)]
    Ds_arr = (ctypes.c_double * max(1, len(Ds_l)))(*Ds_l)
    fn = _entry or LIB.nu_periodic_search
    st = fn(_p(t0s), t0s.numel(), Ds_arr, n_D, _p(depth), _p(var),
                                _p(dlnl), prec, _p(periods), n_P, float(phase_step),
                                float(gap_factor), _stream_ptr(stream), _p(res["Q"]),
                                _p(res["T0"]), _p(res["D_idx"]), _p(res["depth"]),
                                _p(res["sigma"]), _p(res["lnP"]))
    _check(st, "nu_periodic_search")
    return res


def nu_mask_transits(t0s, depth, var, dlnl, period, T0, half_width, precision="fp64",
                     stream=None):
    """Mask, in place, the grid entries within half_width of the transits of
    (period, T0) (see nu_mask_transits in the header); returns the arrays."""
    t0s = _dev(t0s, "t0s")
    dt = torch.float64 if _PREC[precision] == NU_FP64 else torch.float32
    for a, nm in ((depth, "depth"), (var, "var"), (dlnl, "dlnl")):
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == dt
                and a.is_contiguous() and a.numel() % max(1, t0s.numel()) == 0):
            raise ValueError(f"{nm} must be a contiguous CUDA tensor of the precision's dtype "
                             "with n_D * n_t0 elements (masked in place)")
    n_D = depth.numel() // t0s.numel()
    st = LIB.nu_mask_transits(_p(t0s), t0s.numel(), n_D, _p(depth), _p(var), _p(dlnl),
                              _PREC[precision], float(period), float(T0), float(half_width),
                              _stream_ptr(stream))
    _check(st, "nu_mask_transits")
    return depth, var, dlnl


def nu_rotation_alias_filter(periods, P_star, tol=0.02, symmetric=False, stream=None):
    """Period grid without the rotation period's aliases (see
    nu_rotation_alias_filter in the header).  Returns the kept periods (a new
    device tensor; reading its length synchronises the stream)."""
    periods = _dev(periods, "periods")
    kept = torch.empty_like(periods)
    n = torch.empty(1, dtype=torch.int64, device=periods.device)
    st = LIB.nu_rotation_alias_filter(_p(periods), periods.numel(), float(P_star), float(tol),
                                      1 if symmetric else 0, _p(kept), _p(n),
                                      _stream_ptr(stream))
    _check(st, "nu_rotation_alias_filter")
    return kept[: int(n.item())]


def nu_periodic_refine(factor, periods, T0, D_idx, Ds, template="box", ingress_frac=0.1,
                       stream=None, ld=(0.4, 0.25)):
    """Exact periodic-template fit of candidates (see nu_periodic_refine in the
    header).  periods, T0 (float64) and D_idx (int32) are (n_cand,) device
    arrays, e.g. a selection of nu_periodic_search's outputs.  Returns a dict
    of (n_cand,) float64 tensors depth, var, dlnl, snr."""
    periods = _dev(periods, "periods")
    T0 = _dev(T0, "T0")
    D_idx = _dev(D_idx, "D_idx", torch.int32)
    n = periods.numel()
    if T0.numel() != n or D_idx.numel() != n:
        raise ValueError("periods, T0 and D_idx must have the same length")
    Ds_l = [float(d) for d in (Ds.tolist() if hasattr(Ds, "tolist") else Ds)]
    Ds_arr = (ctypes.c_double * max(1, len(Ds_l)))(*Ds_l)
    res = {name: torch.empty(n, dtype=torch.float64, device=periods.device)
           for name in ("depth", "var", "dlnl", "snr")}
    st = LIB.nu_periodic_refine(factor.handle, _p(periods), _p(T0), _p(D_idx), n, Ds_arr,
                                len(Ds_l), _TMPL[template],
                                _tmpl_params(template, ingress_frac, ld),
                                _stream_ptr(stream), _p(res["depth"]), _p(res["var"]),
                                _p(res["dlnl"]), _p(res["snr"]))
    _check(st, "nu_periodic_refine")
    return res


def nu_periodic_search_noalloc(t0s, Ds, depth, var, dlnl, periods, precision="fp64",
                               phase_step=0.0, gap_factor=1.5, stream=None):
    """nu_periodic_search with the library's fixed scratch array (no device
    allocation inside the library call; phase_step must be > 0).  The output
    tensors are still allocated here, by the caller side of the ABI.  The call
    runs with the device of t0s current (the library uses the scratch array
    of the current device and refuses a stream of another device)."""
    with torch.cuda.device(t0s.device):
        return nu_periodic_search(t0s, Ds, depth, var, dlnl, periods, precision=precision,
                                  phase_step=phase_step, gap_factor=gap_factor, stream=stream,
                                  _entry=LIB.nu_periodic_search_noalloc)


def nu_periodic_search_noalloc_limit():
    return int(LIB.nu_periodic_search_noalloc_limit())


def nu_batch_search(curves, Ds, periods, k=2, precision="fp64", phase_step=None,
                    stream=None):
    """Batched search (factor, box linear search with t0 = samples, periodic
    search) of several light curves in one graph launch.

    curves: list of (t, y, diag_var, terms); arrays may be numpy or CUDA
    tensors (float64).  The design matrix of every curve is [1, t][:k].
    phase_step: shared phase step (None or 0: the library takes the median
    sample spacing of the first curve).  Returns a dict of (n_lc, n_P)
    tensors and 'status' (list of per-curve factor statuses, 0 = OK).
    """
    dev = torch.device("cuda", torch.cuda.current_device())
    as_dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev).reshape(-1)
    ts = [as_dev(c[0]) for c in curves]
    t = torch.cat(ts).contiguous()
    y = torch.cat([as_dev(c[1]) for c in curves]).contiguous()
    dv = torch.cat([as_dev(c[2]) for c in curves]).contiguous()
    n_lc = len(curves)
    offs = [0]
    for a in ts:
        offs.append(offs[-1] + a.numel())
    offsets = (ctypes.c_int64 * (n_lc + 1))(*offs)
    flat = [tm for c in curves for tm in c[3]]
    terms = make_terms(flat)
    counts = (ctypes.c_int * n_lc)(*[len(c[3]) for c in curves])
    Ds_l = [float(d) for d in (Ds.tolist() if hasattr(Ds, "tolist") else Ds)]
    Ds_arr = (ctypes.c_double * len(Ds_l))(*Ds_l)
    periods = as_dev(periods).contiguous()
    n_P = periods.numel()
    if phase_step is None:
        phase_step = 0.0
    res = {name: torch.empty((n_lc, n_P), dtype=torch.float64, device=dev)
           for name in ("Q", "T0", "depth", "sigma", "lnP")}
    res["D_idx"] = torch.empty((n_lc, n_P), dtype=torch.int32, device=dev)
    status = (ctypes.c_int * n_lc)()
    st = LIB.nu_batch_search(n_lc, offsets, _p(t), _p(y), _p(dv), terms, counts, int(k),
                             Ds_arr, len(Ds_l), _p(periods), n_P, float(phase_step),
                             _PREC[precision], _stream_ptr(stream), _p(res["Q"]),
                             _p(res["T0"]), _p(res["D_idx"]), _p(res["depth"]),
                             _p(res["sigma"]), _p(res["lnP"]), status)
    _check(st, "nu_batch_search")
    res["status"] = list(status)
    return res


def launch_count():
    """Kernels launched by the library so far (all threads)."""
    return int(LIB.nu_launch_count())


def version():
    return LIB.nu_version().decode()
