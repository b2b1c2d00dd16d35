"""Parity at the two largest benchmark sizes, in the launch configurations
bench.py times.

- The N = 10^8 SEIR job on a random 10-regular graph with BF16 ages (the big
  job of the serving workload; bench.py's `large` block): the graph is built
  on the device as the benchmark builds it, the run goes through CUDA Graph
  replays of 50 steps, the whole trajectory is checked through properties
  that hold at any size (conservation of N, monotone S and R), and a window
  of two steps at the epidemic's growth is lock-stepped against the oracle
  node by node (10^8 nodes per step, from the GPU's own state).
- The 64-graph x 8-scenario packed batch of 500 steps (C3; bench.py's
  `ensemble` block, the same graphs, scenarios, seeds and index cases): every
  one of the 512 realisations keeps N and monotone S and R at every step; a
  sample of realisations spread over the batch equals the same realisation
  run alone, counts bit for bit; and single packed steps of the largest
  graph's ensemble are lock-stepped against the oracle.
"""
import math

import numpy as np
import pytest

import bench
import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import TIE, LockstepReport, ages_as_float, lockstep, oracle_params

pytestmark = pytest.mark.gpu


def test_big_job_n1e8_bf16_sampled_lockstep(oracle_mod):
    import torch
    assert torch.cuda.is_available()
    n, d = 100_000_000, 10
    dev = torch.device("cuda")
    rp, col = bench.device_regular(torch, n, d, seed=0, dev=dev)
    idx = W.index_nodes(n, 100, seed=1)
    p = fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, 1,
                      latent=fs.law("weibull", 2.0, 4.0), age_dtype=fs.FS_AGE_BF16)
    gh = fs.fs_graph_create(n, rp, col, opts=fs.graph_opts(device_input=True))
    s = fs.fs_sim_init(gh, p, idx)
    try:
        counts = fs.fs_sim_run(s, 250, graph_steps=50)
        assert (counts.astype(np.int64).sum(axis=1) == n).all()
        assert (np.diff(counts[:, 0].astype(np.int64)) <= 0).all()
        assert (np.diff(counts[:, 3].astype(np.int64)) >= 0).all()
        assert counts[-1, 1] + counts[-1, 2] > 100_000, "the window must fall in the growth phase"
        g = W.Graph(n, rp.cpu().numpy(), col.cpu().numpy(), "regular10-device")
        del rp, col
        torch.cuda.empty_cache()
        rep = lockstep(oracle_mod, g, p, s, 2, LockstepReport())
        assert rep.decisions > 1_000_000
        assert rep.mismatches <= 1e-6 * rep.decisions
    finally:
        fs.fs_sim_destroy(s)
        fs.fs_graph_destroy(gh)


@pytest.fixture(scope="module")
def c3():
    import torch
    assert torch.cuda.is_available()
    graphs = bench.mixed_graphs(64, 1e4, 2e6, seed=2026)
    assert sum(g.n for g in graphs) > 20_000_000
    ghs = [fs.fs_graph_create(g.n, g.row_ptr, g.col_ind) for g in graphs]
    idxs = [bench.index_for(g, seed=q + 1) for q, g in enumerate(graphs)]
    scen = [W.scenarios(8, seed=1000 + q) for q in range(64)]
    seeds = [int(sc[0].seed) for sc in scen]
    params = [[bench.scen_params(fs, sc, r, fs.FS_AGE_F32, seed=seeds[q]) for r, sc in enumerate(scen[q])]
              for q in range(64)]
    yield graphs, ghs, idxs, params
    for gh in ghs:
        fs.fs_graph_destroy(gh)


def test_c3_packed_batch_full_size(c3):
    graphs, ghs, idxs, params = c3
    steps = 500
    ens = [fs.fs_ens_create(ghs[q], params[q], idxs[q]) for q in range(64)]
    outs = [np.zeros((steps + 1, 8, 4), dtype=np.uint32) for _ in range(64)]
    b = fs.fs_batch_create(fs.FS_AGE_F32, 65)
    try:
        for q in range(64):
            fs.fs_batch_add(b, ens[q], steps, outs[q])
        fs.fs_batch_run(b, steps + 1, 50)
    finally:
        fs.fs_batch_destroy(b)
        for e in ens:
            fs.fs_ens_destroy(e)
    for q, g in enumerate(graphs):
        c = outs[q].astype(np.int64)
        assert (c.sum(axis=2) == g.n).all(), q
        assert (np.diff(c[:, :, 0], axis=0) <= 0).all(), q
        assert (np.diff(c[:, :, 3], axis=0) >= 0).all(), q
    # realisations spread over the batch (graph families, sizes, scenarios)
    # equal their runs alone through the plain engine
    for q in range(0, 64, 7):
        r = q % 8
        s = fs.fs_sim_init(ghs[q], params[q][r], idxs[q])
        alone = fs.fs_sim_run(s, steps, graph_steps=50)
        fs.fs_sim_destroy(s)
        np.testing.assert_array_equal(outs[q][:, r, :], alone, err_msg=f"graph {q} scenario {r}")


def test_c3_largest_graph_packed_lockstep(c3, oracle_mod):
    """Single packed steps of the largest graph's 8-scenario ensemble against
    the oracle, each replicate fed from the ensemble's own state."""
    graphs, ghs, idxs, params = c3
    q = int(np.argmax([g.n for g in graphs]))
    g, ps = graphs[q], params[q]
    e = fs.fs_ens_create(ghs[q], ps, idxs[q])
    decisions = mismatches = 0
    try:
        fs.fs_ens_run(e, 300, 8, 50, want_counts=False)
        for _ in range(2):
            states = [fs.fs_ens_get_state(e, r, g.n) for r in range(8)]
            fs.fs_ens_run(e, 1, 8, 1, want_counts=False)
            for r, p in enumerate(ps):
                X, A, k = states[r]
                Xo, Ao, margin, _ = oracle_mod.step(g.row_ptr, g.col_ind, oracle_params(oracle_mod, p), k, X,
                                                    ages_as_float(A, p.age_dtype), want_margin=True)
                X2, A2, _ = fs.fs_ens_get_state(e, r, g.n)
                decisions += int(np.isfinite(margin).sum())
                bad = X2 != Xo
                assert (np.abs(margin[bad]) < TIE).all(), (r, k, np.flatnonzero(bad)[:8])
                mismatches += int(bad.sum())
                ok = ~bad
                assert (ages_as_float(A2, p.age_dtype)[ok].view(np.uint32) == Ao[ok].view(np.uint32)).all()
        assert decisions > 200_000
        assert mismatches <= 1e-6 * decisions
    finally:
        fs.fs_ens_destroy(e)
