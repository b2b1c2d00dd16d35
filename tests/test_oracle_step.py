"""Pins of the oracle's tau-leaping step (Algorithm 3 at a fixed step;
Section 3 Eqs. 1-3; Section 5.2).

Pins: a brute-force restatement on tiny graphs with uniforms from the
separate numpy Philox; closed-form laws of the discrete scheme (isolated
nodes survive each step with probability exp(-h(a_j) dt); an S-I pair is
infected with a probability given by a one-line dynamic programme; the
exponential case is geometric); conservation and monotonicity invariants;
determinism and exact resumption from a saved state.
"""
import math

import numpy as np
import pytest
import scipy.stats

import workloads as W
from tests import philox_ref

LN5 = math.log(5.0)


def _c0_params(om, seed=1):
    return om.params(om.SIR, None, om.law("lognormal", LN5, 0.5), 0.3, 0.1, seed=seed)


def _seir_params(om, seed=1, age_dtype=0):
    return om.params(om.SEIR, om.law("weibull", 2.0, 4.0), om.law("lognormal", math.log(6), 0.6),
                     0.25, 0.1, seed=seed, age_dtype=age_dtype)


def test_step_matches_brute_force_restatement(oracle_mod):
    """Tiny SEIR graph, every compartment present, ages non-zero: the step is
    recomputed here from the definitions with scipy hazards and numpy Philox."""
    om = oracle_mod
    rng = np.random.default_rng(2)
    n = 60
    g = W.erdos_renyi(n, 6, seed=4)
    prm = _seir_params(om, seed=77)
    for k in (0, 5, 31):
        X = rng.integers(0, 4, n).astype(np.uint8)
        A = np.where((X == 1) | (X == 2), rng.uniform(0, 15, n), 0).astype(np.float32)
        Xn, An, margin, lam = om.step(g.row_ptr, g.col_ind, prm, k, X, A, want_margin=True, want_lambda=True)
        u_all = philox_ref.uniforms(77, 0, k, np.arange(n))
        wb = scipy.stats.weibull_min(c=2.0, scale=4.0)
        ln = scipy.stats.lognorm(s=0.6, scale=6.0)
        for i in range(n):
            x, a = int(X[i]), float(A[i])
            if x == 0:
                c = sum(1 for j in g.col_ind[g.row_ptr[i]:g.row_ptr[i + 1]] if X[j] == 2)
                lmb = 0.25 * c
            elif x == 1:
                lmb = wb.pdf(a) / wb.sf(a) if a > 0 else 0.0
            elif x == 2:
                lmb = ln.pdf(a) / ln.sf(a) if a > 0 else 0.0
            else:
                lmb = 0.0
            assert lam[i] == pytest.approx(lmb, rel=1e-9, abs=1e-300)
            p = 1 - math.exp(-lmb * 0.1)
            fire = p > 0 and u_all[i] < p
            assert Xn[i] == (min(x + 1, 3) if fire else x)
            if fire:
                assert An[i] == 0
            elif x in (1, 2):
                assert An[i] == np.float32(A[i]) + np.float32(0.1)
            else:
                assert An[i] == 0
            if p > 0:
                assert margin[i] == pytest.approx(u_all[i] - p, abs=1e-12)
            else:
                assert margin[i] == np.inf


def test_isolated_nodes_follow_discrete_survival(oracle_mod):
    """Edgeless graph, all nodes I: after k steps the expected fraction still I
    is prod_{j<k} exp(-h(a_j) dt) with a_j the stored age after j steps."""
    om = oracle_mod
    n = 200_000
    g = W.empty_graph(n)
    prm = _c0_params(om, seed=3)
    X, A = om.init(n, np.arange(n), om.I)
    steps = 300
    cnt, _, _ = om.run(g.row_ptr, g.col_ind, prm, 0, steps, X, A)
    ln = scipy.stats.lognorm(s=0.5, scale=5.0)
    a = np.float32(0.0)
    surv = 1.0
    for k in range(steps + 1):
        q = surv
        z = (cnt[k, 2] - n * q) / math.sqrt(n * q * (1 - q) + 1e-12)
        assert abs(z) < 5.0, (k, cnt[k], n * q)
        h = ln.pdf(float(a)) / ln.sf(float(a)) if a > 0 else 0.0
        surv *= math.exp(-h * 0.1)
        a = np.float32(a + np.float32(0.1))
    # the paper's continuous survival at t = 30 differs only by the
    # left-Riemann discretisation of the integrated hazard
    assert abs(cnt[steps, 2] / n - ln.sf(30.0)) < 0.2 * ln.sf(30.0) + 5 * math.sqrt(ln.sf(30.0) / n)


def test_exponential_case_is_geometric(oracle_mod):
    om = oracle_mod
    n = 200_000
    g = W.empty_graph(n)
    prm = om.params(om.SIR, None, om.law("exp", 0.2), 0.3, 0.1, seed=9)
    X, A = om.init(n, np.arange(n), om.I)
    cnt, _, _ = om.run(g.row_ptr, g.col_ind, prm, 0, 100, X, A)
    for k in (1, 10, 50, 100):
        q = math.exp(-0.2 * 0.1 * k)
        z = (cnt[k, 2] - n * q) / math.sqrt(n * q * (1 - q))
        assert abs(z) < 5.0


def test_si_pairs_match_dynamic_programme(oracle_mod):
    """n/2 disjoint S-I pairs: P(S still S after k steps) =
    sum_{m<k} L_m q_m (1-pS)^(m+1) + L_k (1-pS)^k, with q_m the I node's
    recovery probability at step m, L_m = prod_{j<m} (1-q_j), pS = 1-exp(-beta dt)."""
    om = oracle_mod
    pairs = 100_000
    n = 2 * pairs
    u = np.arange(0, n, 2, dtype=np.int64)
    g = W.csr_from_edges(n, u, u + 1)
    beta, dt = 0.05, 0.1
    prm = om.params(om.SIR, None, om.law("lognormal", LN5, 0.5), beta, dt, seed=21)
    X, A = om.init(n, u.astype(np.int32), om.I)
    steps = 200
    Xk = X.copy()
    Ak = A.copy()
    ln = scipy.stats.lognorm(s=0.5, scale=5.0)
    pS = 1 - math.exp(-beta * dt)
    L = 1.0
    acc = 0.0
    a = np.float32(0.0)
    for k in range(steps + 1):
        if k in (1, 20, 80, 200):
            expect = acc + L * (1 - pS) ** k
            still = int((Xk[1::2] == 0).sum())
            z = (still - pairs * expect) / math.sqrt(pairs * expect * (1 - expect))
            assert abs(z) < 5.0, (k, still, pairs * expect)
        h = ln.pdf(float(a)) / ln.sf(float(a)) if a > 0 else 0.0
        q = 1 - math.exp(-h * dt)
        acc += L * q * (1 - pS) ** (k + 1)
        L *= 1 - q
        a = np.float32(a + np.float32(dt))
        if k < steps:
            Xk, Ak, _, _ = om.step(g.row_ptr, g.col_ind, prm, k, Xk, Ak)


def test_invariants_on_parity_workload(oracle_mod):
    om = oracle_mod
    g = W.random_regular(10_000, 10, seed=0)
    idx = W.index_nodes(g.n, 10, seed=1)
    prm = _c0_params(om)
    X, A = om.init(g.n, idx, om.I)
    cnt, Xf, Af = om.run(g.row_ptr, g.col_ind, prm, 0, 300, X, A)
    assert (cnt.sum(axis=1) == g.n).all()
    assert (np.diff(cnt[:, 0].astype(np.int64)) <= 0).all()
    assert (np.diff(cnt[:, 3].astype(np.int64)) >= 0).all()
    assert (cnt[:, 1] == 0).all()
    assert cnt[0].tolist() == [g.n - 10, 0, 10, 0]
    # no compartment is skipped and ages reset on every transition
    Xk, Ak = X, A
    for k in range(60):
        Xn, An, _, _ = om.step(g.row_ptr, g.col_ind, prm, k, Xk, Ak)
        moved = Xn != Xk
        assert ((Xn == Xk) | ((Xk == 0) & (Xn == 2)) | ((Xk == 2) & (Xn == 3))).all()
        assert (An[moved] == 0).all()
        assert (An[(Xn == 0) | (Xn == 3)] == 0).all()
        Xk, Ak = Xn, An


def test_determinism_and_resume(oracle_mod):
    om = oracle_mod
    g = W.barabasi_albert(3000, 3, seed=5)
    idx = W.index_nodes(g.n, 20, seed=2, allowed=W.non_hub_nodes(g))
    prm = _seir_params(om, seed=42)
    X, A = om.init(g.n, idx, om.E)
    c1, X1, A1 = om.run(g.row_ptr, g.col_ind, prm, 0, 300, X, A)
    c2, X2, A2 = om.run(g.row_ptr, g.col_ind, prm, 0, 300, X, A)
    np.testing.assert_array_equal(c1, c2)
    ca, Xa, Aa = om.run(g.row_ptr, g.col_ind, prm, 0, 120, X, A)
    cb, Xb, Ab = om.run(g.row_ptr, g.col_ind, prm, 120, 180, Xa, Aa)
    np.testing.assert_array_equal(np.vstack([ca, cb[1:]]), c1)
    np.testing.assert_array_equal(Xb, X1)
    np.testing.assert_array_equal(Ab.view(np.uint32), A1.view(np.uint32))
    assert c1[-1, 3] > 0 and c1[:, 1].max() > 0


@pytest.mark.parametrize("dtype", [1, 2])
def test_reduced_precision_ages_are_storage_values(oracle_mod, dtype):
    om = oracle_mod
    g = W.random_regular(4000, 8, seed=3)
    idx = W.index_nodes(g.n, 40, seed=5)
    prm = _seir_params(om, seed=8, age_dtype=dtype)
    X, A = om.init(g.n, idx, om.E)
    _, Xf, Af = om.run(g.row_ptr, g.col_ind, prm, 0, 400, X, A)
    if dtype == 1:
        assert (Af.astype(np.float16).astype(np.float32) == Af).all()
    else:
        import torch
        assert (torch.from_numpy(Af).to(torch.bfloat16).float().numpy() == Af).all()
    assert Af.max() > 10
