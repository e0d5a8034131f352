"""Pins of the oracle's covariance (Appendix A, Sect. 3.2) to mathematics.

The SHO covariance of Appendix A is the autocovariance of a damped harmonic
oscillator driven by white noise, so it is fixed uniquely by:
  k(0) = sigma^2, k'(0+) = 0, and k'' + (omega/Q) k' + omega^2 k = 0 for tau > 0.
The tests check those three facts by finite differences on the oracle's
function (a dropped term, a wrong sign or a swapped branch fails one of them),
plus continuity across Q = 1/2 and the closed forms of the rotation map.
"""
import numpy as np
import pytest

from oracle import gp


@pytest.mark.parametrize("Q", [0.2, 0.4, 0.5, 0.7, 3.0, 45.0])
@pytest.mark.parametrize("omega", [0.8, 12.0])
def test_sho_initial_conditions_and_ode(Q, omega):
    sigma = 0.37
    k = lambda tau: gp.sho_kernel(tau, sigma, omega, Q)
    assert k(0.0) == pytest.approx(sigma ** 2, rel=1e-15)
    h = 1e-4 / omega
    # k'(0+) = 0: the one-sided difference is O(h)
    d1 = (k(h) - k(0.0)) / h
    assert abs(d1) < 2.0 * omega ** 2 * sigma ** 2 * h
    # ODE residual at several lags, central differences
    for tau in np.array([0.05, 0.3, 1.1, 2.7]) / omega * 2 * np.pi:
        kp = (k(tau + h) - k(tau - h)) / (2 * h)
        kpp = (k(tau + h) - 2 * k(tau) + k(tau - h)) / (h * h)
        res = kpp + (omega / Q) * kp + omega ** 2 * k(tau)
        scale = omega ** 2 * sigma ** 2
        assert abs(res) < 1e-5 * scale


def test_sho_continuity_across_critical_damping():
    tau = np.linspace(0.0, 3.0, 31)
    crit = gp.sho_kernel(tau, 1.0, 2.0, 0.5)
    below = gp.sho_kernel(tau, 1.0, 2.0, 0.5 - 1e-7)
    above = gp.sho_kernel(tau, 1.0, 2.0, 0.5 + 1e-7)
    np.testing.assert_allclose(below, crit, rtol=0, atol=1e-6)
    np.testing.assert_allclose(above, crit, rtol=0, atol=1e-6)


def test_sho_is_even_in_lag():
    tau = np.linspace(-2.0, 2.0, 9)
    np.testing.assert_array_equal(gp.sho_kernel(tau, 1.0, 3.0, 2.0),
                                  gp.sho_kernel(-tau, 1.0, 3.0, 2.0))


@pytest.mark.parametrize("period,Q0,dQ,f", [(1.0, 5.0, 0.0, 0.5),
                                             (0.3, 0.1, 0.4, 0.2),
                                             (4.0, 20.0, 1.0, 1.5)])
def test_rotation_map_closed_forms(period, Q0, dQ, f):
    sigma = 0.02
    (s1, w1, q1), (s2, w2, q2) = gp.rotation_sho_params(sigma, period, Q0, dQ, f)
    assert q1 == pytest.approx(0.5 + Q0 + dQ)
    assert q2 == pytest.approx(0.5 + Q0)
    assert w2 == pytest.approx(2 * w1)
    # total variance sigma^2 split 1 : f between the modes
    assert s1 ** 2 + s2 ** 2 == pytest.approx(sigma ** 2, rel=1e-14)
    assert s2 ** 2 / s1 ** 2 == pytest.approx(f, rel=1e-14)
    # the primary mode oscillates at exactly the rotation period:
    # its damped angular frequency g*omega/(2Q) equals 2 pi / P
    g1 = np.sqrt(4 * q1 * q1 - 1)
    assert g1 * w1 / (2 * q1) == pytest.approx(2 * np.pi / period, rel=1e-14)
    k = gp.kernel_function([(gp.ROTATION, (sigma, period, Q0, dQ, f, ))])
    assert k(0.0) == pytest.approx(sigma ** 2, rel=1e-14)


def test_exp_term():
    assert gp.exp_kernel(0.0, 2.0, 0.3) == pytest.approx(4.0)
    assert gp.exp_kernel(0.3, 2.0, 0.3) == pytest.approx(4.0 / np.e)
    assert gp.exp_kernel(-0.6, 2.0, 0.3) == pytest.approx(4.0 / np.e ** 2)


def test_covariance_structure():
    rng = np.random.default_rng(1)
    t = np.sort(rng.uniform(0, 3, 40))
    dv = rng.uniform(1e-6, 4e-6, 40)
    terms = [(gp.ROTATION, (1e-2, 0.7, 5.0, 0.0, 0.5)), (gp.EXP, (1e-3, 0.2))]
    S = gp.covariance(t, dv, terms)
    np.testing.assert_array_equal(S, S.T)
    np.testing.assert_allclose(np.diag(S), 1e-4 + 1e-6 + dv, rtol=1e-14)
    np.linalg.cholesky(S)      # positive definite
    # off-diagonal entries are the kernel at the lag
    kf = gp.kernel_function(terms)
    assert S[3, 17] == pytest.approx(float(kf(abs(t[3] - t[17]))), rel=1e-15)


def test_white_noise_only_covariance_is_diagonal():
    t = np.arange(5.0)
    S = gp.covariance(t, np.array([1.0, 2.0, 3.0, 4.0, 5.0]), [])
    np.testing.assert_array_equal(S, np.diag([1.0, 2.0, 3.0, 4.0, 5.0]))
