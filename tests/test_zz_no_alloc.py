"""Allocation-free periodic search (nu_periodic_search_noalloc).

Some callers cannot allocate device memory while they run (a runtime that
reserves all of its memory up front, a plugin whose host forbids allocation
inside a step, a process at its memory limit).  For them the library offers a
periodic search whose scratch is a fixed array inside the library.  These
tests call it through the C ABI and check that two calls in a row give the
same results as nu_periodic_search on the same inputs, for both precisions
and for both fold kernels (regular grid: slot walk; jittered grid: exact
epochs), and that a grid too large for the fixed array is refused.

This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2402_06835_gb300 import synth
from parity import FP64_TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2402_06835_gb300 import api  # noqa: E402


def _grid(jitter, seed=31):
    rng = np.random.default_rng(seed)
    dt = synth.CADENCE_DAYS
    t0s = np.concatenate([np.arange(1500), np.arange(1800, 3600)]) * dt
    t0s = t0s + jitter * dt * rng.uniform(-1, 1, len(t0s)) * (np.arange(len(t0s)) % 4 == 2)
    n = len(t0s)
    g = dict(depth=rng.normal(0, 1e-3, (5, n)), var=rng.uniform(1e-8, 5e-8, (5, n)),
             dlnl=rng.uniform(0, 8, (5, n)))
    g["depth"][3, 700:730] = np.nan
    return t0s, g, dt


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("jitter", [0.0, 0.3])
def test_noalloc_matches_allocating_entry_point(precision, jitter):
    t0s, g, dt = _grid(jitter)
    dty = torch.float64 if precision == "fp64" else torch.float32
    cu = lambda a, d=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=d,
                                                    device="cuda")
    args = (cu(t0s), np.ones(5), cu(g["depth"], dty), cu(g["var"], dty), cu(g["dlnl"], dty),
            cu(np.linspace(0.05, 2.5, 311)))
    ref = api.nu_periodic_search(*args, precision=precision, phase_step=dt)
    for _ in range(2):                      # the fixed array is reused call after call
        got = api.nu_periodic_search_noalloc(*args, precision=precision, phase_step=dt)
        torch.cuda.synchronize()
        assert torch.equal(got["D_idx"], ref["D_idx"])
        for key in ("Q", "T0", "depth", "sigma", "lnP"):
            a, b = got[key].cpu().numpy(), ref[key].cpu().numpy()
            fin = np.isfinite(b)
            assert np.array_equal(np.isfinite(a), fin), key
            err = np.abs(a[fin] - b[fin]) / np.maximum(1.0, np.abs(b[fin]))
            assert err.max(initial=0.0) <= FP64_TOL, (key, err.max())


def test_noalloc_refuses_grids_beyond_its_limit():
    limit = api.nu_periodic_search_noalloc_limit()
    n_D = 8
    n = int(limit // (n_D * 32)) + 1000      # FP64 records alone exceed the limit
    t0s = torch.arange(n, dtype=torch.float64, device="cuda") * synth.CADENCE_DAYS
    z = torch.zeros((n_D, n), dtype=torch.float64, device="cuda")
    with pytest.raises(api.NuanceError) as exc:
        api.nu_periodic_search_noalloc(t0s, np.ones(n_D), z, z + 1e-8, z,
                                       torch.tensor([0.3], dtype=torch.float64, device="cuda"),
                                       phase_step=synth.CADENCE_DAYS)
    assert exc.value.status == api.NU_EINVAL
    assert "scratch" in str(exc.value)


def test_noalloc_requires_explicit_phase_step():
    t0s, g, dt = _grid(0.0)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    with pytest.raises(api.NuanceError):
        api.nu_periodic_search_noalloc(cu(t0s), np.ones(5), cu(g["depth"]), cu(g["var"]),
                                       cu(g["dlnl"]), cu([0.3]), phase_step=0.0)


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs two GPUs")
def test_noalloc_refuses_a_stream_of_another_device():
    """The fixed array of the current device is used; a stream that belongs to
    another device is refused before any work is enqueued."""
    t0s, g, dt = _grid(0.0)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")
    args = (cu(t0s), np.ones(5), cu(g["depth"]), cu(g["var"]), cu(g["dlnl"]), cu([0.3]))
    other = torch.cuda.Stream(device="cuda:1")
    with torch.cuda.device(0), pytest.raises(api.NuanceError) as exc:
        api.nu_periodic_search(*args, phase_step=dt, stream=other,
                               _entry=api.LIB.nu_periodic_search_noalloc)
    assert exc.value.status == api.NU_EINVAL
