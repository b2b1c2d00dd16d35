"""Pins of the oracle's source-node infectivity (Section 5.3, Eq. 8):
rho_j = beta s(tau_j) 1{X_j = I}, with s(tau) the hazard or the density of a
law, stored like an age (fp32, then the storage type), and the pressure of an
S node the sum of the stored rho_j of its infectious in-neighbours (Eq. 3).

- the densities against scipy.stats (textbook pdfs, an independent library);
- s(tau) in both modes against scipy (hazard = pdf / sf);
- the stored value against numpy / torch casts of fp32(beta s);
- a constant profile (the hazard of an exponential law) whose beta s is exact
  in the storage type gives the Markovian-edge trajectory bit for bit;
- a brute-force restatement of whole steps on a tiny graph (scipy profile,
  numpy Philox) in every storage type;
- the explicit infectivity input: the pressure is linear in it.
"""
import math

import numpy as np
import pytest
import scipy.stats
import torch

import workloads as W
from tests import philox_ref

LN5, LN6 = math.log(5.0), math.log(6.0)

LAWS = [
    ("exp", 0.3, 0.0, 0, scipy.stats.expon(scale=1 / 0.3)),
    ("lognormal", LN5, 0.5, 0, scipy.stats.lognorm(s=0.5, scale=5.0)),
    ("lognormal", math.log(4.0), 0.668, 0, scipy.stats.lognorm(s=0.668, scale=4.0)),
    ("weibull", 2.0, 4.0, 0, scipy.stats.weibull_min(c=2.0, scale=4.0)),
    ("weibull", 1.5, 2.0, 0, scipy.stats.weibull_min(c=1.5, scale=2.0)),
    ("erlang", 0.75, 0.0, 3, scipy.stats.gamma(a=3, scale=1 / 0.75)),
    ("erlang", 2.0, 0.0, 7, scipy.stats.gamma(a=7, scale=1 / 2.0)),
]
TAUS = np.concatenate([[0.0, 1e-6, 1e-3, 0.05], np.linspace(0.1, 40.0, 400)])


@pytest.mark.parametrize("kind,a,b,k,ref", LAWS, ids=[f"{L[0]}{i}" for i, L in enumerate(LAWS)])
def test_density_matches_scipy(oracle_mod, kind, a, b, k, ref):
    lw = oracle_mod.law(kind, a, b, k)
    for t in TAUS:
        want = float(ref.pdf(t))
        got = oracle_mod.density(lw, float(t))
        assert got == pytest.approx(want, rel=1e-11, abs=1e-300), (t, got, want)


@pytest.mark.parametrize("kind,a,b,k,ref", LAWS, ids=[f"{L[0]}{i}" for i, L in enumerate(LAWS)])
def test_shedding_modes(oracle_mod, kind, a, b, k, ref):
    om = oracle_mod
    lw = om.law(kind, a, b, k)
    inf = om.law("lognormal", LN5, 0.5)
    p_none = om.params(om.SIR, None, inf, 0.3, 0.1, 1)
    p_haz = om.params(om.SIR, None, inf, 0.3, 0.1, 1, shed_mode=om.SHED_HAZARD, shedding=lw)
    p_den = om.params(om.SIR, None, inf, 0.3, 0.1, 1, shed_mode=om.SHED_DENSITY, shedding=lw)
    for t in TAUS[1:]:
        assert om.shedding(p_none, t) == 1.0
        sf = float(ref.sf(t))
        if sf > 1e-250:
            assert om.shedding(p_haz, t) == pytest.approx(float(ref.pdf(t)) / sf, rel=1e-9)
        assert om.shedding(p_den, t) == pytest.approx(float(ref.pdf(t)), rel=1e-11, abs=1e-300)


@pytest.mark.parametrize("age_dtype", [0, 1, 2])
def test_infectivity_is_stored_like_an_age(oracle_mod, age_dtype):
    om = oracle_mod
    lw = om.law("lognormal", LN5, 0.5)
    beta = 0.37
    prm = om.params(om.SIR, None, lw, beta, 0.1, 1, age_dtype=age_dtype, shed_mode=om.SHED_DENSITY, shedding=lw)
    ref = scipy.stats.lognorm(s=0.5, scale=5.0)
    for t in np.linspace(0.0, 30.0, 301).astype(np.float32):
        r32 = np.float32(beta * float(ref.pdf(float(t))))
        if age_dtype == 0:
            want = r32
        elif age_dtype == 1:
            want = np.float32(np.float16(r32))
        else:
            want = torch.tensor(float(r32), dtype=torch.float32).to(torch.bfloat16).float().item()
        got = om.infectivity(prm, float(t))
        # the oracle's fp64 density and scipy's may round to neighbouring fp32
        # values; the storage cast is then the same unless they straddle a
        # rounding boundary of the storage type
        assert got == want or abs(got - want) <= abs(want) * (2 ** -23 if age_dtype == 0 else 2 ** -7), (t, got, want)


def test_constant_profile_equals_markovian_edges(oracle_mod):
    """s = hazard of Exp(2) = 2 and beta = 0.125: rho = 0.25 exactly in every
    storage type, so the pressure equals the s = 1 run with beta = 0.25."""
    om = oracle_mod
    g = W.random_regular(3000, 8, seed=11)
    idx = W.index_nodes(g.n, 15, seed=12)
    for age_dtype in (0, 2):
        lat, inf = om.law("weibull", 2.0, 4.0), om.law("lognormal", LN6, 0.6)
        base = om.params(om.SEIR, lat, inf, 0.25, 0.1, 5, age_dtype=age_dtype)
        shed = om.params(om.SEIR, lat, inf, 0.125, 0.1, 5, age_dtype=age_dtype, shed_mode=om.SHED_HAZARD,
                         shedding=om.law("exp", 2.0))
        X0, A0 = om.init(g.n, idx, om.E)
        c1, X1, A1 = om.run(g.row_ptr, g.col_ind, base, 0, 300, X0, A0)
        c2, X2, A2 = om.run(g.row_ptr, g.col_ind, shed, 0, 300, X0, A0)
        assert c1[-1, 3] > 100
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_array_equal(X1, X2)
        np.testing.assert_array_equal(A1.view(np.uint32), A2.view(np.uint32))


def _store(x32: np.float32, age_dtype: int) -> float:
    if age_dtype == 0:
        return float(x32)
    if age_dtype == 1:
        return float(np.float32(np.float16(x32)))
    return torch.tensor(float(x32), dtype=torch.float32).to(torch.bfloat16).float().item()


@pytest.mark.parametrize("age_dtype", [0, 1, 2])
@pytest.mark.parametrize("mode", ["hazard", "density"])
def test_step_matches_brute_force_restatement(oracle_mod, age_dtype, mode):
    """Tiny SEIR graph with every compartment present and non-zero ages: the
    step is recomputed from Eqs. 3 and 8 with scipy profiles, storage casts
    from numpy / torch and uniforms from the numpy Philox."""
    om = oracle_mod
    rng = np.random.default_rng(3)
    n, beta, dt = 80, 0.9, 0.1
    g = W.erdos_renyi(n, 7, seed=6)
    lat, inf = om.law("weibull", 2.0, 4.0), om.law("lognormal", LN6, 0.6)
    shed = om.law("lognormal", LN5, 0.5)
    sref = scipy.stats.lognorm(s=0.5, scale=5.0)
    s_of = (lambda t: sref.pdf(t) / sref.sf(t) if t > 0 else 0.0) if mode == "hazard" else sref.pdf
    prm = om.params(om.SEIR, lat, inf, beta, dt, 91, age_dtype=age_dtype,
                    shed_mode=om.SHED_HAZARD if mode == "hazard" else om.SHED_DENSITY, shedding=shed)
    wb = scipy.stats.weibull_min(c=2.0, scale=4.0)
    ln = scipy.stats.lognorm(s=0.6, scale=6.0)
    for k in (0, 9, 40):
        X = rng.integers(0, 4, n).astype(np.uint8)
        X[:20] = 2                                   # plenty of infectious sources
        A = np.where((X == 1) | (X == 2), rng.uniform(0, 15, n), 0).astype(np.float32)
        A = np.array([_store(np.float32(a), age_dtype) for a in A], dtype=np.float32)
        Xn, An, rho_next, margin, lam = om.step_rho(g.row_ptr, g.col_ind, prm, k, X, A)
        u = philox_ref.uniforms(91, 0, k, np.arange(n))
        rho = np.array([_store(np.float32(beta * float(s_of(float(a)))), age_dtype) if x == 2 else 0.0
                        for x, a in zip(X, A)])
        n_src = 0
        for i in range(n):
            x, a = int(X[i]), float(A[i])
            if x == 0:
                row = g.col_ind[g.row_ptr[i]:g.row_ptr[i + 1]]
                lmb = float(sum(rho[j] for j in row if X[j] == 2))
                n_src += int(any(X[j] == 2 for j in row))
            elif x == 1:
                lmb = wb.pdf(a) / wb.sf(a) if a > 0 else 0.0
            elif x == 2:
                lmb = ln.pdf(a) / ln.sf(a) if a > 0 else 0.0
            else:
                lmb = 0.0
            assert lam[i] == pytest.approx(lmb, rel=1e-9, abs=1e-300), (k, i, x)
            p = 1 - math.exp(-lmb * dt)
            fire = p > 0 and u[i] < p
            assert Xn[i] == (min(x + 1, 3) if fire else x)
            if Xn[i] == 2:
                want = _store(np.float32(beta * float(s_of(float(An[i])))), age_dtype)
                assert rho_next[i] == pytest.approx(want, rel=2.0 ** -22, abs=1e-300)
            else:
                assert rho_next[i] == 0.0
        assert n_src > 5


def test_explicit_infectivity_input(oracle_mod):
    """rho_in replaces the computed infectivities: equal inputs give the
    same step, doubled inputs double every S pressure, and non-I entries are
    never read."""
    om = oracle_mod
    g = W.erdos_renyi(500, 6, seed=8)
    rng = np.random.default_rng(9)
    shed = om.law("lognormal", LN5, 0.5)
    prm = om.params(om.SIR, None, om.law("lognormal", LN5, 0.5), 0.4, 0.1, 3, shed_mode=om.SHED_DENSITY,
                    shedding=shed)
    X = rng.choice([0, 2, 3], 500, p=[0.6, 0.3, 0.1]).astype(np.uint8)
    A = np.where(X == 2, rng.uniform(0, 12, 500), 0).astype(np.float32)
    rho = np.array([om.infectivity(prm, float(a)) if x == 2 else 0.0 for x, a in zip(X, A)], dtype=np.float32)
    r0 = om.step_rho(g.row_ptr, g.col_ind, prm, 4, X, A)
    r1 = om.step_rho(g.row_ptr, g.col_ind, prm, 4, X, A, rho_in=rho)
    for a, b in zip(r0, r1):
        np.testing.assert_array_equal(a, b)
    junk = np.where(X == 2, 2 * rho, 1e6).astype(np.float32)
    r2 = om.step_rho(g.row_ptr, g.col_ind, prm, 4, X, A, rho_in=junk)
    S = X == 0
    np.testing.assert_allclose(r2[4][S], 2 * r0[4][S], rtol=1e-15)
    np.testing.assert_array_equal(r2[4][~S], r0[4][~S])


def test_exact_simulator_rejects_shedding(oracle_mod):
    om = oracle_mod
    g = W.random_regular(50, 4, seed=1)
    prm = om.params(om.SIR, None, om.law("exp", 0.2), 0.3, 0.1, 1, shed_mode=om.SHED_DENSITY,
                    shedding=om.law("lognormal", LN5, 0.5))
    with pytest.raises(ValueError):
        om.exact_run(g.row_ptr, g.col_ind, prm, [1], om.I, 5, 10, 1.0)


def test_constant_profile_adaptive_equals_markovian_edges(oracle_mod):
    """The adaptive step (Section 5.2) with the exact constant profile: the
    pressure, lambda*, every dt_k and the trajectory equal the s = 1 run."""
    om = oracle_mod
    g = W.random_regular(2000, 8, seed=13)
    idx = W.index_nodes(g.n, 20, seed=14)
    lat, inf = om.law("weibull", 2.0, 4.0), om.law("lognormal", LN6, 0.6)
    base = om.params(om.SEIR, lat, inf, 0.25, 0.1, 7)
    shed = om.params(om.SEIR, lat, inf, 0.125, 0.1, 7, shed_mode=om.SHED_HAZARD, shedding=om.law("exp", 2.0))
    X0, A0 = om.init(g.n, idx, om.E)
    c1, X1, A1, d1, l1 = om.run_adaptive(g.row_ptr, g.col_ind, base, 0.03, 1e-12, 0, 400, X0, A0)
    c2, X2, A2, d2, l2 = om.run_adaptive(g.row_ptr, g.col_ind, shed, 0.03, 1e-12, 0, 400, X0, A0)
    assert d1.min() < 0.1 and c1[-1, 3] > 50
    np.testing.assert_array_equal(d1, d2)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(A1.view(np.uint32), A2.view(np.uint32))
    assert l1 == l2
