"""The injection-recovery workload follows the set-up it stands in for
(Sect. 3, first comparison, and Eq. relative_params)."""
import numpy as np

from paper_2402_06835_gb300 import synth


def test_injection_workload_parameters():
    w = synth.injection_4000(n_curves=50)
    assert len(w.curves) == 50 and list(w.durations) == [0.04]
    assert w.periods[0] == 0.3 and w.periods[-1] == 3.0 and len(w.periods) == 4000
    for lc in w.curves:
        assert len(lc.t) == 2880 and lc.t[-1] < 4.0
        (kind, (sigma, omega, q, _, _)), = lc.terms
        inj = lc.injected
        assert kind == synth.TERM_SHO
        # Eq. relative_params: tau = pi / (omega D), delta = 2 sigma / depth
        assert abs(np.pi / (omega * 0.04) - inj["tau"]) < 1e-12 * inj["tau"]
        assert abs(2 * sigma / 0.01 - inj["delta"]) < 1e-12 * inj["delta"]
        assert 0.1 <= inj["tau"] <= 10 and 0.1 <= inj["delta"] <= 25 and 10 <= q <= 100
        assert np.all(lc.diag_var == 1e-6)
    # a quiet curve shows the four 1 % dips at 0.2 + 1.1 k
    quiet = min(w.curves, key=lambda lc: lc.injected["delta"])
    t, y = quiet.t, quiet.y
    for tc in (0.2, 1.3, 2.4, 3.5):
        inside = np.abs(t - tc) < 0.015
        around = (np.abs(t - tc) > 0.03) & (np.abs(t - tc) < 0.08)
        assert y[around].mean() - y[inside].mean() > 0.007
