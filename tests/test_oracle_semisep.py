"""Pins of the sequential celerite reference (oracle/semisep.py) to the dense
oracle: the same log-determinant, solves and per-template GLS on light
curves where the dense matrix fits."""
import numpy as np
import pytest

from oracle import gp, linear, semisep
from paper_2402_06835_gb300 import synth


def test_semisep_matches_dense_covariance_solves():
    lc = synth.small_curve(n=400, seed=13, gap=60)
    terms = lc.terms + [(gp.EXP, (3e-3, 0.1))]
    ss = semisep.Semisep(lc.t, lc.diag_var, terms)
    dense = linear.DenseModel(lc.t, lc.y, lc.diag_var, terms, lc.X)
    assert ss.logdet == pytest.approx(dense.logdet, rel=1e-12)
    # y^T Sigma^-1 y from the innovations equals the dense whitened norm
    e = ss.innovations(lc.y[:, None])[:, 0]
    assert float(e @ (e / ss.D)) == pytest.approx(float(dense.yw @ dense.yw), rel=1e-10)


@pytest.mark.parametrize("kind", ["box", "trapezoid"])
def test_semisep_templates_match_dense_oracle(kind):
    lc = synth.small_curve(n=600, seed=17, gap=45)
    Ds = np.array([0.02, 0.06])
    rng = np.random.default_rng(1)
    pairs = [(int(rng.integers(0, 2)), int(i)) for i in rng.integers(0, len(lc.t), 40)]
    pairs += [(1, 0), (0, len(lc.t) - 1), (1, 299), (1, 300)]
    d, v, l, model = semisep.sampled_linear_search(lc.t, lc.y, lc.diag_var, lc.terms, lc.X,
                                                   Ds, pairs, kind=kind, ingress_frac=0.2)
    dense = linear.DenseModel(lc.t, lc.y, lc.diag_var, lc.terms, lc.X)
    dd, dv, dl = linear.sampled_linear_search(dense, lc.t, Ds, pairs, kind=kind,
                                              ingress_frac=0.2)
    sd = np.sqrt(dv)
    assert np.max(np.abs(d - dd) / np.maximum(np.abs(dd), sd)) < 1e-10
    assert np.max(np.abs(v - dv) / dv) < 1e-10
    assert np.max(np.abs(l - dl) / np.maximum(dl, 1.0)) < 1e-9
    assert model.lnL_null == pytest.approx(dense.lnL_null, rel=1e-12)
