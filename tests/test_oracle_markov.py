"""Pins of the oracle's Markovian engine (Section 4, Algorithm 1) and of its
exact Doob-Gillespie reference.

- Gillespie against the exact continuous-time Markov chain of a 5-node graph
  (all 2^5 SIS / 3^5 SIR configurations; transient law by a matrix
  exponential of the generator): mean counts at 9 times.
- Algorithm 1 with small steps against the same matrix exponential.
- A brute-force restatement of single steps (numpy rates and tau, numpy
  Philox) for SIS, SIR and SEIR.
- The tau rule in closed form; isolated SIS nodes recover to S with
  probability 1 - exp(-gamma tau) (z-test).
- The paper's validation protocol (Erdos-Renyi N = 10^3, d = 8, beta = 0.25,
  recovery 0.15, 10 seeds, 100 runs, max_prob 0.1, theta 0.01): the
  tau-leaping mean lies inside the exact simulator's 25-75% band at every one
  of 100 grid times, for SIS and SIR.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from tests import philox_ref

S, E, I, R = 0, 1, 2, 3


def small_graph():
    """5 nodes: a ring plus two chords (undirected)."""
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 2), (3, 1)]
    return W.csr_from_edges(5, np.array([a for a, _ in edges]), np.array([b for _, b in edges]))


def ctmc_mean_counts(g, model, beta, gamma, index, times, sigma=0.0):
    """Exact E[#S], E[#I], E[#R] (and E[#E] last for SEIR) of the Markov
    chain at the given times."""
    n = g.n
    comps = {"sis": (S, I), "sir": (S, I, R), "seir": (S, E, I, R)}[model]
    states = list(itertools.product(comps, repeat=n))
    pos = {s: q for q, s in enumerate(states)}
    Q = np.zeros((len(states), len(states)))
    for s in states:
        a = pos[s]
        for i in range(n):
            if s[i] == S:
                c = sum(1 for j in g.col_ind[g.row_ptr[i]:g.row_ptr[i + 1]] if s[j] == I)
                rate, y = beta * c, (E if model == "seir" else I)
            elif s[i] == E:
                rate, y = sigma, I
            elif s[i] == I:
                rate, y = gamma, (S if model == "sis" else R)
            else:
                continue
            if rate > 0:
                t = list(s)
                t[i] = y
                Q[a, pos[tuple(t)]] += rate
                Q[a, a] -= rate
    p0 = np.zeros(len(states))
    p0[pos[tuple(I if i in index else S for i in range(n))]] = 1.0
    cnt = np.array([[sum(1 for x in s if x == c) for c in (S, I, R, E)] for s in states], dtype=float)
    return np.array([(p0 @ scipy.linalg.expm(Q * t)) @ cnt for t in times])


@pytest.mark.parametrize("model", ["sis", "sir"])
def test_gillespie_matches_exact_chain(oracle_mod, model):
    om = oracle_mod
    g = small_graph()
    beta, gamma = 0.9, 0.6
    prm = om.params(om.SIS if model == "sis" else om.SIR, None, om.law("exp", gamma), beta, 0.1, 1)
    times = np.arange(9) * 0.5
    exact = ctmc_mean_counts(g, model, beta, gamma, {0}, times)
    runs = np.array([om.gillespie_run(g.row_ptr, g.col_ind, prm, [0], om.I, 1000 + r, 9, 0.5)
                     for r in range(20_000)], dtype=float)
    for col, c in ((0, S), (1, I), (2, R)):
        if model == "sis" and c == R:
            continue
        m = runs[:, :, c].mean(axis=0)
        se = runs[:, :, c].std(axis=0) / math.sqrt(runs.shape[0])
        assert (np.abs(m - exact[:, col]) <= 4.5 * se + 1e-9).all(), (c, m, exact[:, col], se)


@pytest.mark.parametrize("model", ["sis", "sir"])
def test_small_steps_converge_to_exact_chain(oracle_mod, model):
    om = oracle_mod
    g = small_graph()
    beta, gamma = 0.9, 0.6
    times = np.arange(9) * 0.5
    exact = ctmc_mean_counts(g, model, beta, gamma, {0}, times)
    X0, A0 = om.init(g.n, [0], om.I)
    acc = []
    for r in range(4000):
        prm = om.params(om.SIS if model == "sis" else om.SIR, None, om.law("exp", gamma), beta, 0.1, 77 + r)
        cnt, _, _, _ = om.markov_run(g.row_ptr, g.col_ind, prm, 1e-3, 0.005, 0.005, 0, 9, 0.5, X0, A0)
        acc.append(cnt)
    runs = np.array(acc, dtype=float)
    m = runs[:, :, I].mean(axis=0)
    se = runs[:, :, I].std(axis=0) / math.sqrt(runs.shape[0])
    # statistical error plus the scheme's O(p_max) bias (the step is at most
    # 0.005 d; grid times are matched to the step boundary at or before them)
    assert (np.abs(m - exact[:, 1]) <= 4.5 * se + 0.02).all(), (m, exact[:, 1], se)


def numpy_tau(g, X, beta, sigma, gamma, theta, p_max, tau_max):
    si = ne = ni = cmax = 0
    for i in range(g.n):
        if X[i] == S:
            c = int(np.sum(X[g.col_ind[g.row_ptr[i]:g.row_ptr[i + 1]]] == I))
            si += c
            cmax = max(cmax, c)
        elif X[i] == E:
            ne += 1
        elif X[i] == I:
            ni += 1
    lam = beta * si + sigma * ne + gamma * ni
    lmax = beta * cmax
    if ne and sigma > lmax:
        lmax = sigma
    if ni and gamma > lmax:
        lmax = gamma
    tau = tau_max
    if lam > 0 and theta * g.n / lam < tau:
        tau = theta * g.n / lam
    if lmax > 0 and p_max / lmax < tau:
        tau = p_max / lmax
    return np.float32(tau), lam, lmax


@pytest.mark.parametrize("model", ["sis", "sir", "seir"])
def test_step_matches_brute_force_restatement(oracle_mod, model):
    om = oracle_mod
    rng = np.random.default_rng(4)
    g = W.erdos_renyi(70, 6, seed=3)
    beta, sigma, gamma = 0.7, 0.4, 0.3
    code = {"sis": om.SIS, "sir": om.SIR, "seir": om.SEIR}[model]
    prm = om.params(code, om.law("exp", sigma) if model == "seir" else None, om.law("exp", gamma), beta, 0.1, 55)
    states = {"sis": [S, I], "sir": [S, I, R], "seir": [S, E, I, R]}[model]
    for k, theta, p_max in ((0, 0.01, 0.1), (6, 0.5, 0.1), (21, 0.05, 0.9)):
        X = rng.choice(states, g.n).astype(np.uint8)
        A = np.where((X == E) | (X == I), rng.uniform(0, 9, g.n), 0).astype(np.float32)
        tau_np, lam_np, lmax_np = numpy_tau(g, X, beta, sigma if model == "seir" else 0.0, gamma, theta, p_max, 0.1)
        tau, lam, lmax = om.markov_tau(g.row_ptr, g.col_ind, prm, theta, p_max, 0.1, X)
        assert tau == tau_np and lam == pytest.approx(lam_np, rel=1e-15) and lmax == lmax_np
        Xn, An, margin, tau_used = om.markov_step(g.row_ptr, g.col_ind, prm, theta, p_max, 0.1, k, X, A)
        assert tau_used == tau
        u = philox_ref.uniforms(55, 0, k, np.arange(g.n))
        for i in range(g.n):
            x = int(X[i])
            if x == S:
                lmb = beta * int(np.sum(X[g.col_ind[g.row_ptr[i]:g.row_ptr[i + 1]]] == I))
            elif x == E:
                lmb = sigma
            elif x == I:
                lmb = gamma
            else:
                lmb = 0.0
            p = -math.expm1(-lmb * float(tau))
            fire = p > 0 and u[i] < p
            nxt = {S: E if model == "seir" else I, E: I, I: S if model == "sis" else R}
            assert Xn[i] == (nxt[x] if fire else x), (k, i, x)
            if fire:
                assert An[i] == 0
            elif x in (E, I):
                assert An[i] == np.float32(A[i]) + np.float32(tau)
            if p > 0:
                assert margin[i] == pytest.approx(u[i] - p, abs=1e-12)
            else:
                assert margin[i] == np.inf


def test_tau_rule_closed_forms(oracle_mod):
    om = oracle_mod
    n = 100
    g = W.empty_graph(n)
    prm = om.params(om.SIS, None, om.law("exp", 0.5), 0.3, 0.1, 1)
    X = np.zeros(n, dtype=np.uint8)
    assert om.markov_tau(g.row_ptr, g.col_ind, prm, 0.01, 0.1, 0.25, X) == (np.float32(0.25), 0.0, 0.0)
    X[:] = I                                    # Lambda = 50, max lambda = 0.5
    for theta, p_max, tmax in ((0.01, 0.1, 1.0), (1.0, 0.1, 1.0), (1.0, 0.9, 1.0), (1.0, 0.9, 0.3)):
        tau, lam, lmax = om.markov_tau(g.row_ptr, g.col_ind, prm, theta, p_max, tmax, X)
        assert lam == 50.0 and lmax == 0.5
        assert tau == np.float32(min(theta * n / 50.0, p_max / 0.5, tmax))


def test_isolated_sis_nodes_recover_to_s(oracle_mod):
    om = oracle_mod
    n = 200_000
    g = W.empty_graph(n)
    prm = om.params(om.SIS, None, om.law("exp", 0.7), 0.3, 0.1, 9)
    X = np.full(n, I, dtype=np.uint8)
    A = np.zeros(n, dtype=np.float32)
    Xn, _, _, tau = om.markov_step(g.row_ptr, g.col_ind, prm, 1.0, 0.2, 1.0, 3, X, A)
    assert tau == np.float32(0.2 / 0.7)
    assert set(np.unique(Xn)) <= {S, I}
    p = -math.expm1(-0.7 * float(tau))
    k = int(np.sum(Xn == S))
    assert abs(k - n * p) <= 4.5 * math.sqrt(n * p * (1 - p))


@pytest.mark.parametrize("model", ["sis", "sir"])
def test_papers_validation_protocol(oracle_mod, model):
    om = oracle_mod
    g = W.erdos_renyi(1000, 8, seed=21)
    idx = W.index_nodes(g.n, 10, seed=22)
    code = om.SIS if model == "sis" else om.SIR
    n_grid, grid_dt, runs = 100, 0.4, 100
    exact = np.array([om.gillespie_run(g.row_ptr, g.col_ind, om.params(code, None, om.law("exp", 0.15), 0.25, 0.1, 1),
                                       idx, om.I, 5000 + r, n_grid, grid_dt)[:, I] for r in range(runs)], dtype=float)
    X0, A0 = om.init(g.n, idx, om.I)
    tl = np.array([om.markov_run(g.row_ptr, g.col_ind, om.params(code, None, om.law("exp", 0.15), 0.25, 0.1, 900 + r),
                                 0.01, 0.1, 0.1, 0, n_grid, grid_dt, X0, A0)[0][:, I] for r in range(runs)],
                  dtype=float)
    q25, q75 = np.percentile(exact, 25, axis=0), np.percentile(exact, 75, axis=0)
    mean = tl.mean(axis=0)
    assert ((mean >= q25) & (mean <= q75)).all(), np.flatnonzero((mean < q25) | (mean > q75))
    assert exact.mean(axis=0).max() > 100          # a real outbreak (SIR peak, SIS endemic level)


def test_seir_gillespie_and_small_steps_match_exact_chain(oracle_mod):
    """SEIR with exponential latent and infectious periods (4^5 states)."""
    om = oracle_mod
    g = small_graph()
    beta, sigma, gamma = 0.9, 0.8, 0.6
    times = np.arange(9) * 0.5
    exact = ctmc_mean_counts(g, "seir", beta, gamma, {0}, times, sigma=sigma)
    prm = om.params(om.SEIR, om.law("exp", sigma), om.law("exp", gamma), beta, 0.1, 1)
    gil = np.array([om.gillespie_run(g.row_ptr, g.col_ind, prm, [0], om.I, 3000 + r, 9, 0.5)
                    for r in range(20_000)], dtype=float)
    X0, A0 = om.init(g.n, [0], om.I)
    tl = np.array([om.markov_run(g.row_ptr, g.col_ind,
                                 om.params(om.SEIR, om.law("exp", sigma), om.law("exp", gamma), beta, 0.1, 500 + r),
                                 1e-3, 0.005, 0.005, 0, 9, 0.5, X0, A0)[0] for r in range(4000)], dtype=float)
    for col, c in ((1, I), (2, R), (3, E)):
        m = gil[:, :, c].mean(axis=0)
        se = gil[:, :, c].std(axis=0) / math.sqrt(gil.shape[0])
        assert (np.abs(m - exact[:, col]) <= 4.5 * se + 1e-9).all(), ("gillespie", c, m, exact[:, col])
        m = tl[:, :, c].mean(axis=0)
        se = tl[:, :, c].std(axis=0) / math.sqrt(tl.shape[0])
        assert (np.abs(m - exact[:, col]) <= 4.5 * se + 0.02).all(), ("tau-leap", c, m, exact[:, col])


def test_gillespie_agrees_with_the_event_driven_simulator(oracle_mod):
    """SIR with exponential recovery: the Doob-Gillespie run and the oracle's
    event-driven renewal simulator (holding times drawn at entry) simulate
    the same process by different algorithms; their mean trajectories agree."""
    om = oracle_mod
    g = W.erdos_renyi(200, 6, seed=8)
    idx = W.index_nodes(g.n, 5, seed=9)
    prm = om.params(om.SIR, None, om.law("exp", 0.2), 0.3, 0.1, 1)
    a = np.array([om.gillespie_run(g.row_ptr, g.col_ind, prm, idx, om.I, 11 + r, 31, 1.0)
                  for r in range(1500)], dtype=float)
    b = np.array([om.exact_run(g.row_ptr, g.col_ind, prm, idx, om.I, 7001 + r, 31, 1.0)
                  for r in range(1500)], dtype=float)
    for c in (I, R):
        d = a[:, :, c].mean(axis=0) - b[:, :, c].mean(axis=0)
        se = np.sqrt(a[:, :, c].var(axis=0) / a.shape[0] + b[:, :, c].var(axis=0) / b.shape[0])
        assert (np.abs(d) <= 4.5 * se + 1e-9).all(), (c, d, se)
    assert a[:, -1, R].mean() > 50
