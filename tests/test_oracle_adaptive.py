"""Pins of the oracle's adaptive step (Section 5.2): dt_k = min(dt_max,
eps / (lambda*_{k-1} + delta)), lambda* the largest rate of the previous step,
dt_max at the first step.

- With an eps that never binds the adaptive run is the fixed-step run.
- The step size follows the rule with lambda* recomputed independently from
  the state (numpy pressure counts, scipy hazards).
- Exponential recovery on isolated nodes is a Markov chain: the survivors
  after K adaptive steps are binomial with p = prod exp(-gamma dt_j).
- On the paper's validation benchmark the adaptive ensembles at eps = 0.03 and
  0.1 match its printed tau-leap values (Table "Convergence sweep").
"""
import math
import os

import numpy as np
import scipy.stats

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "epsilon_sweep.txt")
DELTA = 1e-12


def seir(om, beta=0.25, dt=0.1, seed=3):
    return om.params(om.SEIR, om.law("weibull", 2.0, 4.0), om.law("lognormal", math.log(6.0), 0.6), beta, dt,
                     seed=seed)


def test_unbinding_eps_equals_fixed_step(oracle_mod):
    om = oracle_mod
    g = W.random_regular(2000, 6, seed=4)
    idx = W.index_nodes(g.n, 20, seed=5)
    prm = seir(om)
    X0, A0 = om.init(g.n, idx, om.E)
    c_fix, X_fix, A_fix = om.run(g.row_ptr, g.col_ind, prm, 0, 250, X0, A0)
    c_ad, X_ad, A_ad, dts, _ = om.run_adaptive(g.row_ptr, g.col_ind, prm, 1e9, DELTA, 0, 250, X0, A0)
    np.testing.assert_array_equal(c_ad, c_fix)
    np.testing.assert_array_equal(X_ad, X_fix)
    np.testing.assert_array_equal(A_ad.view(np.uint32), A_fix.view(np.uint32))
    assert np.all(dts == np.float32(0.1))


def rates_independent(g, X, A, beta, lat, inf_mu, inf_sigma):
    """lambda_i from the state: beta x (# I in-neighbours) for S, Weibull and
    log-normal hazards (scipy pdf / sf) for E and I, 0 for R."""
    isI = (X == 2).astype(np.int64)
    c = np.add.reduceat(isI[g.col_ind], g.row_ptr[:-1]) if g.nnz else np.zeros(g.n, np.int64)
    c[np.diff(g.row_ptr) == 0] = 0
    lam = np.zeros(g.n)
    lam[X == 0] = beta * c[X == 0]
    tE = A[X == 1].astype(np.float64)
    k, s = lat
    lam[X == 1] = (k / s) * (tE / s) ** (k - 1)
    tI = A[X == 2].astype(np.float64)
    d = scipy.stats.lognorm(inf_sigma, scale=math.exp(inf_mu))
    with np.errstate(divide="ignore", invalid="ignore"):
        h = np.where(tI > 0, d.pdf(tI) / d.sf(tI), 0.0)
    lam[X == 2] = h
    return lam


def test_step_size_follows_the_rule(oracle_mod):
    om = oracle_mod
    g = W.erdos_renyi(400, 6, seed=7)
    idx = W.index_nodes(g.n, 8, seed=8)
    eps = 0.03
    prm = seir(om, beta=0.4, dt=0.1, seed=9)
    X, A = om.init(g.n, idx, om.E)
    lam_prev = 0.0
    bound_hits = 0
    for k in range(400):
        lam = rates_independent(g, X, A, 0.4, (2.0, 4.0), math.log(6.0), 0.6)
        _, X, A, dts, lam_last = om.run_adaptive(g.row_ptr, g.col_ind, prm, eps, DELTA, k, 1, X, A, lam_prev)
        # this step's size came from the previous step's largest rate
        want = np.float32(min(0.1, eps / (lam_prev + DELTA)))
        assert abs(float(dts[0]) - float(want)) <= 2 * np.spacing(want)
        assert float(dts[0]) <= min(0.1, eps / (lam_prev + DELTA)) * (1 + 1e-7)
        # and this step's largest rate is the independent maximum
        assert math.isclose(lam_last, float(lam.max()), rel_tol=1e-9, abs_tol=1e-300)
        bound_hits += float(dts[0]) < 0.1
        lam_prev = lam_last
    assert bound_hits > 50                  # the bound binds for much of the run


def test_isolated_exponential_nodes_follow_the_product_law(oracle_mod):
    om = oracle_mod
    n, gamma, eps = 200_000, 0.5, 0.02
    g = W.empty_graph(n)
    prm = om.params(om.SIR, None, om.law("exp", gamma), 0.3, 0.1, seed=11)
    X, A = om.init(n, np.arange(n, dtype=np.int32), om.I)
    cnt, _, _, dts, _ = om.run_adaptive(g.row_ptr, g.col_ind, prm, eps, DELTA, 0, 60, X, A)
    assert float(dts[0]) == np.float32(0.1)
    assert np.all(dts[1:] == np.float32(eps / (gamma + DELTA)))
    for k in (10, 30, 60):
        q = math.exp(-gamma * float(np.sum(dts[:k].astype(np.float64))))
        mean, sd = n * q, math.sqrt(n * q * (1 - q))
        assert abs(int(cnt[k, 2]) - mean) <= 5 * sd


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[f[0]] = tuple(float(x) for x in f[1:])
    return rows


def test_eps_sweep_matches_the_papers_tau_leap_values(oracle_mod):
    """ER N = 1000, d = 8, beta = 0.25, log-normal E->I (mean 5, median 4) and
    I->R (mean 7.5, median 5), 10 index E, T = 50 d, tau_max = 0.1, 100 runs."""
    om = oracle_mod
    g = W.erdos_renyi(1000, 8, seed=0)
    sE = math.sqrt(2 * math.log(5 / 4))
    sI = math.sqrt(2 * math.log(7.5 / 5))
    gold = _golden()
    for eps in ("0.03", "0.1"):
        pk, fr = [], []
        for r in range(100):
            prm = om.params(om.SEIR, om.law("lognormal", math.log(4), sE), om.law("lognormal", math.log(5), sI),
                            0.25, 0.1, seed=7000 + r)
            X, A = om.init(g.n, W.index_nodes(g.n, 10, seed=100 + r), om.E)
            t, lam, k, peak = 0.0, 0.0, 0, 0
            while t < 50.0:
                cnt, X, A, dts, lam = om.run_adaptive(g.row_ptr, g.col_ind, prm, float(eps), DELTA, k, 1, X, A,
                                                      lam)
                t += float(dts[0])
                k += 1
                peak = max(peak, int(cnt[1, 2]))
            pk.append(peak / g.n)
            fr.append(int(cnt[1, 3]) / g.n)
        ci = lambda x: 1.96 * np.std(x) / math.sqrt(len(x))
        row = gold[eps]
        assert abs(np.mean(pk) - row[0]) <= 3 * row[1] + ci(pk), (eps, np.mean(pk), row)
        assert abs(np.mean(fr) - row[2]) <= 3 * row[3] + ci(fr), (eps, np.mean(fr), row)
