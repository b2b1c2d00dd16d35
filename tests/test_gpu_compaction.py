"""Active-node compaction (Section 5.6, FS_ACTIVE_LIST) on the GPU.

R is absorbing, so visiting only the units (SELL slices, push items) that
held a non-R node at the start of a launch sequence cannot change a
trajectory: with and without the list, counts, states and ages agree bit for
bit (the paper checks compartment counts at five checkpoints; these tests
check every step's counts and the final state). Each case runs past the point
where half the nodes are R, so the list is in use (fs_sim_active_units shows
fewer units visited than without it); cases cover both pressure forms, the
shared-memory and the global-bitmap gather kernels, the push kernel's
one-item-per-lane and block-scan instances, graph replays and directly
launched remainders, a shedding profile and the adaptive step. With the list
in use, single steps are also checked against the oracle itself (lock-step:
each step from the GPU's own state), in both pressure forms.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import lockstep

pytestmark = pytest.mark.gpu

LN6 = math.log(6.0)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fs.load()
    return torch


def seir(pressure, seed=3, **kw):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 0.25, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), pressure=pressure, **kw)


def paired_run(gh, n, p, idx, steps, graph_steps, set_state=None):
    """The same run without and with FS_ACTIVE_LIST; returns both results."""
    out = []
    for flag in (0, fs.FS_ACTIVE_LIST):
        q = fs.sim_params(p.model, p.infectious, p.beta, p.dt, p.seed, latent=p.latent, age_dtype=p.age_dtype,
                          pressure=p.flags | flag, eps=p.eps, delta=p.delta, shed_mode=p.shed_mode,
                          shedding=p.shedding)
        s = fs.fs_sim_init(gh, q, idx)
        if set_state is not None:
            fs.fs_sim_set_state(s, *set_state)
        c = fs.fs_sim_run(s, steps, graph_steps=graph_steps)
        X, A, k = fs.fs_sim_get_state(s, n, p.age_dtype)
        listed, units = fs.fs_sim_active_units(s)
        t = fs.fs_sim_time(s)[0]
        out.append((c, X, A, listed, units, t))
        fs.fs_sim_destroy(s)
    return out


def assert_same_and_listed(res, sequences):
    (c0, X0, A0, l0, u0, t0), (c1, X1, A1, l1, u1, t1) = res
    np.testing.assert_array_equal(c0, c1)
    np.testing.assert_array_equal(X0, X1)
    np.testing.assert_array_equal(A0.view(np.uint8), A1.view(np.uint8))
    assert t0 == t1
    assert u0 == 0 and l0 == 0
    assert u1 > 0 and l1 < sequences * u1, (l1, sequences, u1)
    assert c1[-1, 3] * 2 > X1.size


@pytest.mark.parametrize("pressure", [fs.FS_PRESSURE_GATHER, fs.FS_PRESSURE_PUSH], ids=["gather", "push"])
@pytest.mark.parametrize("graph_steps", [50, 7], ids=["K50", "K7"])
def test_ba_saturating_run_identical(torch_cuda, pressure, graph_steps):
    g = W.barabasi_albert(50_003, 4, seed=7)
    idx = W.index_nodes(g.n, 50, seed=2, allowed=W.non_hub_nodes(g))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    steps = 703
    res = paired_run(gh, g.n, seir(pressure), idx, steps, graph_steps)
    assert_same_and_listed(res, steps // graph_steps + (steps % graph_steps > 0))
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", [fs.FS_PRESSURE_GATHER, fs.FS_PRESSURE_PUSH], ids=["gather", "push"])
def test_regular_thread_class_only(torch_cuda, pressure):
    g = W.random_regular(40_000, 10, seed=1)
    idx = W.index_nodes(g.n, 40, seed=5)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    res = paired_run(gh, g.n, seir(pressure, seed=9), idx, 800, 50)
    assert_same_and_listed(res, 16)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", [fs.FS_PRESSURE_GATHER, fs.FS_PRESSURE_PUSH], ids=["gather", "push"])
def test_large_graph_global_bitmap_and_block_scan(torch_cuda, pressure):
    """N = 1.7 * 10^6 from a mostly-recovered state (R 80%): the gather form's
    SELL class runs in the fused grid (the bitmap exceeds shared memory) and
    the push kernel in its block-scan instance; the list is used at once."""
    n = 1_700_000
    g = W.random_regular(n, 6, seed=4)
    rng = np.random.default_rng(8)
    X = rng.choice([fs.FS_S, fs.FS_E, fs.FS_I, fs.FS_R], n, p=[0.1, 0.05, 0.05, 0.8]).astype(np.uint8)
    A = np.where((X == fs.FS_E) | (X == fs.FS_I), rng.uniform(0, 12, n), 0).astype(np.float32)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    res = paired_run(gh, n, seir(pressure, seed=12), [0], 120, 50, set_state=(X, A, 31))
    assert_same_and_listed(res, 3)
    fs.fs_graph_destroy(gh)


def test_with_shedding_profile(torch_cuda):
    g = W.barabasi_albert(30_011, 4, seed=3)
    idx = W.index_nodes(g.n, 60, seed=4, allowed=W.non_hub_nodes(g))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    p = seir(fs.FS_PRESSURE_AUTO, seed=5, shed_mode=fs.FS_SHED_HAZARD, shedding=fs.law("exp", 2.0))
    res = paired_run(gh, g.n, p, idx, 650, 50)
    assert_same_and_listed(res, 13)
    fs.fs_graph_destroy(gh)


def test_with_adaptive_step(torch_cuda):
    g = W.random_regular(30_000, 8, seed=6)
    idx = W.index_nodes(g.n, 30, seed=7)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    p = seir(fs.FS_PRESSURE_PUSH, seed=6, eps=0.2)
    res = paired_run(gh, g.n, p, idx, 1500, 50)
    assert_same_and_listed(res, 30)
    fs.fs_graph_destroy(gh)


def test_compaction_argument_errors(torch_cuda):
    g = W.random_regular(300, 4, seed=1)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    bad = seir(fs.FS_PRESSURE_PUSH)
    bad.flags = fs.FS_PRESSURE_PUSH | 0x8
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, bad, [1])
    assert e.value.status == 1
    bad.flags = 3
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, bad, [1])
    assert e.value.status == 1
    with pytest.raises(fs.FsError) as e:
        fs.fs_ens_create(gh, [seir(fs.FS_PRESSURE_AUTO | fs.FS_ACTIVE_LIST, seed=k) for k in range(3)], [1])
    assert e.value.status == 7
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", [fs.FS_PRESSURE_GATHER, fs.FS_PRESSURE_PUSH], ids=["gather", "push"])
def test_listed_steps_lockstep_with_oracle(torch_cuda, oracle_mod, pressure):
    """Past the point where half the nodes are R (step ~260 here; the oracle's
    own run has R = 39,931 of 50,003 at step 300), every single step opens a
    launch sequence whose refresh lists the live units, and the listed sweep's
    next state equals the oracle's step from the same state."""
    g = W.barabasi_albert(50_003, 4, seed=7)
    idx = W.index_nodes(g.n, 50, seed=2, allowed=W.non_hub_nodes(g))
    p = seir(pressure | fs.FS_ACTIVE_LIST)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    c = fs.fs_sim_run(s, 280, graph_steps=50)
    assert c[-1, 3] * 2 > g.n
    l0, u = fs.fs_sim_active_units(s)
    rep = lockstep(oracle_mod, g, p, s, 40)
    l1, _ = fs.fs_sim_active_units(s)
    assert rep.decisions > 100_000
    assert l1 - l0 < 40 * u, "the refreshes of the 40 single steps must list fewer than all units"
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
