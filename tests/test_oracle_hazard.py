"""Pins of the oracle's double-precision hazards (Section 5.1, Proposition 1).

The hazard of every law is checked against its definition h = f/S with the
density f and survival S taken from libraries that know nothing of erfcx
(mpmath at 40 digits, scipy.stats), against closed forms, and against the
limits the paper states (h -> 0 as tau -> 0 after a reset, Appendix A).
erfcx itself is checked on the paper's validation grid z in [-9, 30] with
10,001 points (Appendix A) against mpmath's exp(z^2) erfc(z) at 40 digits.
"""
import math
from fractions import Fraction

import mpmath
import numpy as np
import pytest
import scipy.special
import scipy.stats

mpmath.mp.dps = 40


def test_erfcx_on_paper_grid_against_mpmath(oracle_mod):
    zs = np.linspace(-9.0, 30.0, 10001)
    worst = 0.0
    for z in zs:
        ref = mpmath.exp(mpmath.mpf(z) ** 2) * mpmath.erfc(mpmath.mpf(z))
        got = oracle_mod.erfcx(float(z))
        worst = max(worst, abs(got - float(ref)) / float(ref))
    assert worst < 2e-13


def test_erfcx_identities(oracle_mod):
    assert oracle_mod.erfcx(0.0) == pytest.approx(1.0, rel=1e-15)
    for z in (0.3, 1.7, 4.0, 8.5):
        # reflection erfcx(-z) = 2 exp(z^2) - erfcx(z)   (Appendix A)
        assert oracle_mod.erfcx(-z) == pytest.approx(2 * math.exp(z * z) - oracle_mod.erfcx(z), rel=1e-13)
    for z in (30.0, 100.0, 1e4, 1e8):
        # asymptote z sqrt(pi) erfcx(z) -> 1
        assert z * math.sqrt(math.pi) * oracle_mod.erfcx(z) == pytest.approx(1.0 - 1 / (2 * z * z) + 3 / (4 * z**4), rel=1e-8)
    for z in (-3.0, 0.5, 2.0, 25.0, 27.0, 40.0):
        # erfcx'(z) = 2 z erfcx(z) - 2/sqrt(pi), by a central difference
        h = 1e-5 * max(1.0, abs(z))
        d = (oracle_mod.erfcx(z + h) - oracle_mod.erfcx(z - h)) / (2 * h)
        assert d == pytest.approx(2 * z * oracle_mod.erfcx(z) - 2 / math.sqrt(math.pi), rel=1e-5, abs=1e-9)
    # scipy's independent erfcx
    for z in np.linspace(-20, 60, 801):
        assert oracle_mod.erfcx(float(z)) == pytest.approx(float(scipy.special.erfcx(z)), rel=1e-13)


def _ln_hazard_mp(tau, mu, sigma):
    tau = mpmath.mpf(tau)
    x = (mpmath.log(tau) - mu) / sigma
    f = mpmath.exp(-x * x / 2) / (tau * sigma * mpmath.sqrt(2 * mpmath.pi))
    S = mpmath.erfc(x / mpmath.sqrt(2)) / 2
    return f / S


@pytest.mark.parametrize("mu,sigma", [(math.log(5), 0.5), (math.log(6), 0.6), (math.log(4), 0.668),
                                      (math.log(5), 0.901), (math.log(6), 0.3), (math.log(6), 1.0)])
def test_lognormal_hazard_equals_density_over_survival(oracle_mod, mu, sigma):
    law = oracle_mod.law("lognormal", mu, sigma)
    for tau in [1e-3, 0.05, 0.1, 0.5, 1, 2, 5, 10, 30, 60, 100, 300]:
        ref = float(_ln_hazard_mp(tau, mpmath.mpf(mu), mpmath.mpf(sigma)))
        got = oracle_mod.hazard(law, tau)
        if ref < 1e-300:
            assert got < 1e-290
        else:
            assert got == pytest.approx(ref, rel=1e-12)


def test_lognormal_values_and_limits(oracle_mod):
    law = oracle_mod.law("lognormal", math.log(5), 0.5)
    # independent values from scipy.stats (pdf / sf)
    d = scipy.stats.lognorm(s=0.5, scale=5.0)
    for tau in (1.0, 5.0, 30.0):
        assert oracle_mod.hazard(law, tau) == pytest.approx(d.pdf(tau) / d.sf(tau), rel=1e-9)
    assert oracle_mod.hazard(law, 0.0) == 0.0                 # h(0) = 0 (Appendix A)
    assert oracle_mod.hazard(law, 1e-300) == 0.0              # z -> -inf: underflows to 0
    # long-tau behaviour of the log-normal hazard: ~ (ln tau - mu)/(sigma^2 tau)
    tau = 1e12
    x = (math.log(tau) - math.log(5)) / 0.5
    assert oracle_mod.hazard(law, tau) == pytest.approx(x / (0.5 * tau), rel=0.02)


def test_weibull_erlang_exponential_closed_forms(oracle_mod):
    w = oracle_mod.law("weibull", 2.0, 4.0)
    for tau in (0.0, 0.1, 1.0, 3.7, 20.0):
        assert oracle_mod.hazard(w, tau) == pytest.approx(tau / 8.0, rel=1e-15, abs=0)
    w3 = oracle_mod.law("weibull", 1.5, 2.0)
    d = scipy.stats.weibull_min(c=1.5, scale=2.0)
    for tau in (0.2, 1.0, 5.0):
        assert oracle_mod.hazard(w3, tau) == pytest.approx(d.pdf(tau) / d.sf(tau), rel=1e-12)
    w1 = oracle_mod.law("weibull", 1.0, 4.0)
    assert oracle_mod.hazard(w1, 0.0) == 0.25                 # k = 1 is exponential
    e = oracle_mod.law("erlang", 0.75, k=3)
    # Erlang(3, r=0.75) at tau = 1: exact rational arithmetic
    x = Fraction(3, 4)
    exact = Fraction(3, 4) * (x * x / 2) / (1 + x + x * x / 2)
    assert oracle_mod.hazard(e, 1.0) == pytest.approx(float(exact), rel=1e-15)
    assert oracle_mod.hazard(e, 0.0) == 0.0
    g = scipy.stats.gamma(a=3, scale=1 / 0.75)
    for tau in (0.3, 2.0, 9.0, 40.0):
        assert oracle_mod.hazard(e, tau) == pytest.approx(g.pdf(tau) / g.sf(tau), rel=1e-10)
    assert oracle_mod.hazard(e, 1e4) == pytest.approx(0.75, rel=1e-3)   # -> r
    ex = oracle_mod.law("exp", 0.2)
    for tau in (0.0, 1.0, 100.0):
        assert oracle_mod.hazard(ex, tau) == 0.2


def test_hazard_is_minus_log_survival_derivative(oracle_mod):
    """h = -d/dtau ln S(tau), S from mpmath, for every law (catches a dropped
    factor anywhere in a hazard formula)."""
    cases = [
        (oracle_mod.law("lognormal", math.log(6), 0.6),
         lambda t: mpmath.erfc((mpmath.log(t) - mpmath.log(6)) / (mpmath.mpf("0.6") * mpmath.sqrt(2))) / 2),
        (oracle_mod.law("weibull", 2.0, 4.0), lambda t: mpmath.exp(-(t / 4) ** 2)),
        (oracle_mod.law("erlang", 0.75, k=3),
         lambda t: mpmath.exp(-0.75 * t) * (1 + 0.75 * t + (0.75 * t) ** 2 / 2)),
        (oracle_mod.law("exp", 0.3), lambda t: mpmath.exp(-0.3 * t)),
    ]
    for lw, S in cases:
        for tau in (0.4, 2.5, 7.0, 15.0):
            ref = -mpmath.diff(lambda t: mpmath.log(S(t)), mpmath.mpf(tau))
            assert oracle_mod.hazard(lw, tau) == pytest.approx(float(ref), rel=1e-10)
