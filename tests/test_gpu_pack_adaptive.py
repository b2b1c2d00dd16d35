"""The adaptive step (Section 5.2) inside packed ensembles and the server.

Each realisation of an ensemble keeps its own step size, dt_k = min(dt_max,
eps / (lambda*_{k-1} + delta)) with lambda* the largest rate of that
realisation in its previous step, and its own clock. So every packed
realisation must reproduce, bit for bit, the run it has alone through
fs_sim_* (counts every step, final states and ages, elapsed time, next step
size), in both pressure forms and through the hub rows of a Barabasi-Albert
graph; and single packed steps must agree with the oracle run for exactly the
GPU's dt_k of each realisation (lock-step, mismatches only in the near-tie
band, ages bit for bit where states agree). Served requests with eps > 0 equal
their realisations alone.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import TIE, ages_as_float, oracle_params

pytestmark = pytest.mark.gpu

LN6 = math.log(6.0)
DT_REL = 2e-5


def seir(beta, seed, replicate=0, eps=0.03, pressure=fs.FS_PRESSURE_AUTO, sigma=0.6):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, sigma), beta, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), replicate=replicate, eps=eps, pressure=pressure)


def realisations(pressure):
    """8 realisations: four sharing a key (replicates 0..3, one Philox call
    serves them in the packed step) and four with keys of their own."""
    out = [seir(0.25 + 0.05 * r, seed=77, replicate=r, pressure=pressure) for r in range(4)]
    out += [seir(0.15 + 0.1 * r, seed=900 + r, replicate=0, pressure=pressure, sigma=0.4 + 0.1 * r)
            for r in range(4)]
    return out


@pytest.fixture(scope="module")
def ba():
    import torch
    assert torch.cuda.is_available()
    g = W.barabasi_albert(30_000, 4, seed=21)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    assert fs.fs_graph_info_get(gh)["n_merge"] > 0
    idx = W.index_nodes(g.n, 30, seed=3, allowed=W.non_hub_nodes(g))
    yield g, gh, idx
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", [fs.FS_PRESSURE_GATHER, fs.FS_PRESSURE_PUSH], ids=["gather", "push"])
def test_adaptive_ensemble_equals_each_realisation_alone(ba, pressure):
    g, gh, idx = ba
    params = realisations(pressure)
    steps = 300
    e = fs.fs_ens_create(gh, params, idx)
    try:
        _check_alone(g, gh, idx, params, steps, e)
    finally:
        fs.fs_ens_destroy(e)


def _check_alone(g, gh, idx, params, steps, e):
    counts = fs.fs_ens_run(e, steps, len(params), 50)
    t_ens, dt_ens = fs.fs_ens_time(e, len(params))
    for r, p in enumerate(params):
        s = fs.fs_sim_init(gh, p, idx)
        c = fs.fs_sim_run(s, steps)
        t, dt_next = fs.fs_sim_time(s)
        X, A, _ = fs.fs_sim_get_state(s, g.n)
        fs.fs_sim_destroy(s)
        np.testing.assert_array_equal(counts[:, r, :], c, err_msg=f"realisation {r}")
        Xe, Ae, _ = fs.fs_ens_get_state(e, r, g.n)
        np.testing.assert_array_equal(Xe, X)
        np.testing.assert_array_equal(Ae.view(np.uint32), A.view(np.uint32))
        assert t_ens[r] == t and dt_ens[r] == np.float32(dt_next), (r, t_ens[r], t, dt_ens[r], dt_next)
    # the rule bound: some realisation's step fell below dt_max at some point
    assert (t_ens < steps * 0.1 - 1e-9).any()


def test_adaptive_ensemble_lockstep_with_oracle(ba, oracle_mod):
    g, gh, idx = ba
    om = oracle_mod
    params = realisations(fs.FS_PRESSURE_AUTO)[2:6]     # two sharing a key, two with their own
    e = fs.fs_ens_create(gh, params, idx)
    try:
        _lockstep(g, om, params, e)
    finally:
        fs.fs_ens_destroy(e)


def _lockstep(g, om, params, e):
    fs.fs_ens_run(e, 120, len(params), 50, want_counts=False)     # into the epidemic
    decisions = mismatches = 0
    shrunk = False
    for _ in range(15):
        _, dts = fs.fs_ens_time(e, len(params))
        prev = []
        for r, p in enumerate(params):
            prev.append(fs.fs_ens_get_state(e, r, g.n))
        fs.fs_ens_run(e, 1, len(params), 1, want_counts=False)
        for r, p in enumerate(params):
            X, A, k = prev[r]
            prm = oracle_params(om, p)
            prm.dt = float(dts[r])
            shrunk |= bool(dts[r] < np.float32(p.dt))
            Xo, Ao, margin, lam = om.step(g.row_ptr, g.col_ind, prm, k, X, A, want_margin=True, want_lambda=True)
            X2, A2, _ = fs.fs_ens_get_state(e, r, g.n)
            bad = X2 != Xo
            trials = np.isfinite(margin)
            decisions += int(trials.sum())
            if bad.any():
                assert (np.abs(margin[bad]) < TIE).all(), (r, k, margin[bad][:10])
                mismatches += int(bad.sum())
            ok = ~bad
            assert (A2[ok].view(np.uint32) == Ao[ok].view(np.uint32)).all(), (r, k)
            # the next step's size against the oracle's rule on its own rates
            dt_ref = om.adaptive_dt(p.dt, p.eps, 1e-12, float(lam.max()) if lam.size else 0.0)
            _, dts_next = fs.fs_ens_time(e, len(params))
            assert abs(dts_next[r] - dt_ref) <= DT_REL * dt_ref, (r, k, dts_next[r], dt_ref)
    assert mismatches <= 1e-6 * decisions and decisions > 50_000, (mismatches, decisions)
    assert shrunk, "eps must bind in this window"


def test_served_adaptive_request_equals_alone(ba):
    g, gh, idx = ba
    scen = [seir(0.3, seed=41, replicate=0), seir(0.2, seed=41, replicate=3)]
    srv = fs.fs_server_create(quantum=5)
    try:
        rid = fs.fs_server_submit(srv, gh, scen, 3, idx, 150)
        fs.fs_server_drain(srv, 300)
        done, c, _ = fs.fs_server_poll(srv, rid, 150, 6)
        assert done
        for j, p in enumerate(scen):
            for r in range(3):
                q = seir(p.beta, seed=p.seed, replicate=p.replicate + r)
                s = fs.fs_sim_init(gh, q, idx)
                ref = fs.fs_sim_run(s, 150)
                fs.fs_sim_destroy(s)
                np.testing.assert_array_equal(c[:, j * 3 + r, :], ref, err_msg=f"scenario {j} replicate {r}")
    finally:
        fs.fs_server_destroy(srv)


def test_batch_mixes_fixed_and_adaptive_ensembles(ba):
    """One segment table holding fixed-step and adaptive ensembles of both
    pressure forms: each kind runs its own kernel instance, and every
    realisation still equals its run alone."""
    g, gh, idx = ba
    steps = 200
    kinds = [(fs.FS_PRESSURE_GATHER, 0.0), (fs.FS_PRESSURE_PUSH, 0.0),
             (fs.FS_PRESSURE_GATHER, 0.03), (fs.FS_PRESSURE_PUSH, 0.03)]
    sets = [[seir(0.2 + 0.05 * r, seed=300 + j, replicate=r, eps=eps, pressure=pr) for r in range(6)]
            for j, (pr, eps) in enumerate(kinds)]
    ens = [fs.fs_ens_create(gh, ps, idx) for ps in sets]
    b = fs.fs_batch_create(fs.FS_AGE_F32, len(ens))
    try:
        outs = [np.zeros((steps + 1, 6, 4), dtype=np.uint32) for _ in ens]
        for e, o in zip(ens, outs):
            fs.fs_batch_add(b, e, steps, o)
        fs.fs_batch_run(b, steps + 1, 50)
        for j, ps in enumerate(sets):
            for r, p in enumerate(ps):
                s = fs.fs_sim_init(gh, p, idx)
                ref = fs.fs_sim_run(s, steps)
                fs.fs_sim_destroy(s)
                np.testing.assert_array_equal(outs[j][:, r, :], ref, err_msg=f"kind {kinds[j]} realisation {r}")
        t, _ = fs.fs_ens_time(ens[3], 6)
        assert (t < steps * 0.1 - 1e-9).any()
    finally:
        fs.fs_batch_destroy(b)
        for e in ens:
            fs.fs_ens_destroy(e)
