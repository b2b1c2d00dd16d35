"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (device-resident CSR ingest, CUDA Graph replays of 50 steps): the
10-regular SEIR workload and the Barabasi-Albert (m = 5) workload, N = 10^6,
1,000 steps.

At this size the oracle checks sampled windows of ten steps one by one
(lock-step from the GPU's own state: from the start, in the growth phase,
around the peak, in the decline and in the tail), and the whole
trajectory is checked through properties that hold at any size:
conservation of N, monotone S and R, no compartment skipped, and equality of
the graph-replayed run with the same run from a checkpoint.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import LockstepReport, lockstep

pytestmark = pytest.mark.gpu


def seir(seed=1):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0))


@pytest.mark.parametrize("kind", ["regular", "ba"])
def test_full_size_sampled_lockstep(oracle_mod, kind):
    import torch
    assert torch.cuda.is_available()
    n = 1_000_000
    if kind == "regular":
        g = W.random_regular(n, 10, seed=0)
        idx = W.index_nodes(n, 100, seed=1)
    else:
        g = W.barabasi_albert(n, 5, seed=0)
        idx = W.index_nodes(n, 100, seed=1, allowed=W.non_hub_nodes(g))
    d_rp = torch.from_numpy(g.row_ptr).cuda()
    d_col = torch.from_numpy(g.col_ind).cuda()
    gh = fs.fs_graph_create(n, d_rp, d_col, opts=fs.graph_opts(device_input=True))
    info = fs.fs_graph_info_get(gh)
    assert fs.fs_graph_info(gh) == info
    if kind == "ba":
        assert info["n_merge"] > 0 and info["d_max"] > 1000
    p = seir()
    # the whole trajectory in the benchmark configuration
    s = fs.fs_sim_init(gh, p, idx)
    counts = fs.fs_sim_run(s, 1000, graph_steps=50)
    assert (counts.sum(axis=1) == n).all()
    assert (np.diff(counts[:, 0].astype(np.int64)) <= 0).all()
    assert (np.diff(counts[:, 3].astype(np.int64)) >= 0).all()
    assert counts[-1, 3] > n // 2
    Xf, Af, kf = fs.fs_sim_get_state(s, n)
    fs.fs_sim_destroy(s)
    # sampled lock-step: windows of 10 steps from the start, in the growth
    # phase, around the peak, and in the decline and the tail
    peak = int(np.argmax(counts[:, 2]))
    s = fs.fs_sim_init(gh, p, idx)
    rep = LockstepReport()
    done = 0
    for at in sorted({0, 120, max(peak - 5, 10), 450, 700, 900}):
        if at < done:
            continue
        if at > done:
            fs.fs_sim_run(s, at - done, graph_steps=50, want_counts=False)
            done = at
        lockstep(oracle_mod, g, p, s, 10, rep)
        done += 10
    fs.fs_sim_run(s, 1000 - done, graph_steps=50, want_counts=False)
    X2, A2, k2 = fs.fs_sim_get_state(s, n)
    assert k2 == kf == 1000
    if rep.mismatches == 0:
        np.testing.assert_array_equal(X2, Xf)
        np.testing.assert_array_equal(A2.view(np.uint32), Af.view(np.uint32))
    assert rep.decisions > 1_000_000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
