"""Plain FP64 CPU oracle for the nuance hot path (arXiv:2402.06835).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library in ``paper_2402_06835_gb300`` never imports it and has
no CPU fallback: the oracle exists to check the CUDA path, not to stand in
for it.

It is written from the paper's definitions, in the paper's order, with numpy
and scipy's LAPACK routines as the only library steps:

* ``gp``        the SHO kernel of Appendix A, the rotation kernel map and the
                exponential terms of Sect. 3.2 ("Stellar variability kernel"),
                and the dense covariance matrix (white noise on the diagonal).
* ``linear``    the linear search of Sect. 2.2: one generalised least-squares
                fit (Eq. ls) per (epoch, duration) with the log-likelihood of
                Eq. linear_search_ll, on the dense covariance.
* ``periodic``  the periodic search of Sect. 2.3-2.4: interpolation onto the
                phase grid, the combination of Eq. result with the biased
                estimates of Eq. sigma_delta, the argmax of Eq. phi0 and
                Q(P) = Delta/sigma.
* ``semisep``   a second, sequential FP64 reference for light curves too long
                for the dense matrix: the celerite semiseparable Cholesky of
                the same covariance, pinned to ``linear`` where both run.

Nothing here shares code with the CUDA sources; the two meet only through the
seeded inputs of ``paper_2402_06835_gb300.synth``.
"""
from . import gp, linear, periodic, refine, semisep  # noqa: F401
