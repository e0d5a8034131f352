"""nuance (arXiv:2402.06835) hot path on GB300: linear search and periodic fold.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/nuance.h``); ``api`` is its thin binding.  The binding is imported on
first use of one of its names so that ``synth`` (input generation) works on a
machine without the library.
"""
_API_NAMES = ("nu_gp_factor", "nu_factor_info", "nu_linear_search",
              "nu_periodic_search", "nu_batch_search", "NuanceError", "Factor")


def __getattr__(name):
    if name in _API_NAMES:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
