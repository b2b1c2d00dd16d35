"""Packed ensembles and batches against realisations run alone.

Packing changes the layout and the launch, not the arithmetic: every
realisation of an ensemble (its own beta, laws, seed and replicate index)
must produce exactly the counts and the final state it produces alone
through fs_sim_*, whatever the number of replicates (padding to 8, 16 or 32
lanes), the graph (regular, or Barabasi-Albert with hub rows), the age
storage, and whether the ensemble runs alone, in a batch with others, or
joins a batch that is already running, and in both forms of the pressure
(push and gather), also mixed in one batch. One small
ensemble is also compared with the oracle directly.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available()
    fs.load()
    return torch


PRESSURES = [pytest.param(fs.FS_PRESSURE_PUSH, id="push"), pytest.param(fs.FS_PRESSURE_GATHER, id="gather")]


def scenarios(R, seed0=100, age_dtype=fs.FS_AGE_F32, pressure=fs.FS_PRESSURE_AUTO):
    """R realisations with different betas, infectious sigmas and latent laws."""
    rng = np.random.default_rng(seed0)
    out = []
    for r in range(R):
        beta = float(rng.uniform(0.1, 0.5))
        sig = float(rng.uniform(0.3, 1.0))
        latent = fs.law("erlang", 0.75, k=3) if r % 2 == 0 else fs.law("weibull", 2.0, 4.0)
        out.append(fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), sig), beta, 0.1,
                                 seed=seed0 + 7 * r, latent=latent, replicate=r, age_dtype=age_dtype,
                                 pressure=pressure))
    return out


def alone(gh, n, p, idx, steps, age_dtype=fs.FS_AGE_F32):
    s = fs.fs_sim_init(gh, p, idx)
    c = fs.fs_sim_run(s, steps)
    X, A, _ = fs.fs_sim_get_state(s, n, age_dtype)
    fs.fs_sim_destroy(s)
    return c, X, A


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("kind,R,age_dtype", [("regular", 5, fs.FS_AGE_F32), ("regular", 12, fs.FS_AGE_F32),
                                              ("ba", 32, fs.FS_AGE_F32), ("ba", 8, fs.FS_AGE_F16),
                                              ("er", 16, fs.FS_AGE_BF16)])
def test_ensemble_equals_each_realisation_alone(cuda, kind, R, age_dtype, pressure):
    if kind == "regular":
        g = W.random_regular(20_003 + 1, 10, seed=2)
    elif kind == "ba":
        g = W.barabasi_albert(30_001, 4, seed=4)
    else:
        g = W.erdos_renyi(25_000, 8, seed=6)
    idx = W.index_nodes(g.n, 40, seed=3, allowed=W.non_hub_nodes(g) if kind == "ba" else None)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    if kind == "ba":
        assert fs.fs_graph_info_get(gh)["n_merge"] > 0
    ps = scenarios(R, age_dtype=age_dtype, pressure=pressure)
    steps = 220
    e = fs.fs_ens_create(gh, ps, idx)
    c_ens = fs.fs_ens_run(e, steps, R, graph_steps=50)
    for r in range(R):
        c, X, A = alone(gh, g.n, ps[r], idx, steps, age_dtype)
        np.testing.assert_array_equal(c_ens[:, r, :], c, err_msg=f"replicate {r}")
        Xe, Ae, ke = fs.fs_ens_get_state(e, r, g.n, age_dtype)
        assert ke == steps
        np.testing.assert_array_equal(Xe, X)
        np.testing.assert_array_equal(Ae.view(np.uint8), A.view(np.uint8))
    assert c_ens[-1, :, 3].max() > 0
    fs.fs_ens_destroy(e)
    fs.fs_graph_destroy(gh)


def test_batch_members_join_leave_and_resume(cuda):
    """Three ensembles on three graphs join a running batch at different
    launches with different lengths; each member's counts equal its
    realisations alone; an ensemble that left can continue alone. The first
    member pushes, the Barabasi-Albert member gathers and the third takes the
    default form (the gather at 32 replicate lanes), so one launch steps
    segments of both forms."""
    graphs = [W.random_regular(8_000, 6, seed=11), W.barabasi_albert(12_000, 3, seed=12),
              W.erdos_renyi(9_000, 8, seed=13)]
    ghs = [fs.fs_graph_create(g.n, g.row_ptr, g.col_ind) for g in graphs]
    idxs = [W.index_nodes(g.n, 20, seed=21 + q) for q, g in enumerate(graphs)]
    Rs = [12, 3, 20]          # all three replicate widths (16, 8, 32 lanes)
    forms = [fs.FS_PRESSURE_PUSH, fs.FS_PRESSURE_GATHER, fs.FS_PRESSURE_AUTO]
    params = [scenarios(R, seed0=500 + 100 * q, pressure=forms[q]) for q, R in enumerate(Rs)]
    ens = [fs.fs_ens_create(ghs[q], params[q], idxs[q]) for q in range(3)]
    steps = [150, 90, 120]
    outs = [np.zeros((steps[q] + 1, Rs[q], 4), dtype=np.uint32) for q in range(3)]
    b = fs.fs_batch_create(fs.FS_AGE_F32, 16)
    fs.fs_batch_add(b, ens[0], steps[0], outs[0])
    fs.fs_batch_run(b, 40, graph_steps=16)
    fs.fs_batch_add(b, ens[1], steps[1], outs[1])
    fs.fs_batch_run(b, 33, graph_steps=16)
    fs.fs_batch_add(b, ens[2], steps[2], outs[2])
    while True:
        live, need = fs.fs_batch_status(b)
        if live == 0:
            break
        fs.fs_batch_run(b, max(1, min(need, 37)), graph_steps=16)
    fs.fs_batch_destroy(b)
    for q in range(3):
        for r in range(Rs[q]):
            c, X, A = alone(ghs[q], graphs[q].n, params[q][r], idxs[q], steps[q])
            np.testing.assert_array_equal(outs[q][:, r, :], c, err_msg=f"member {q} replicate {r}")
            Xe, Ae, ke = fs.fs_ens_get_state(ens[q], r, graphs[q].n)
            assert ke == steps[q]
            np.testing.assert_array_equal(Xe, X)
            np.testing.assert_array_equal(Ae.view(np.uint32), A.view(np.uint32))
    # member 0 continues alone for 60 more steps: equals 210 steps in one go
    more = fs.fs_ens_run(ens[0], 60, Rs[0], graph_steps=25)
    for r in range(Rs[0]):
        c, _, _ = alone(ghs[0], graphs[0].n, params[0][r], idxs[0], steps[0] + 60)
        np.testing.assert_array_equal(more[:, r, :], c[steps[0]:], err_msg=f"resumed replicate {r}")
    for e in ens:
        fs.fs_ens_destroy(e)
    for gh in ghs:
        fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
def test_small_ensemble_matches_oracle(cuda, oracle_mod, pressure):
    g = W.barabasi_albert(3_000, 3, seed=8)
    idx = W.index_nodes(g.n, 15, seed=9, allowed=W.non_hub_nodes(g))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(thread_max_deg=31))
    ps = scenarios(6, seed0=900, pressure=pressure)
    e = fs.fs_ens_create(gh, ps, idx)
    c_ens = fs.fs_ens_run(e, 200, 6)
    for r in range(6):
        X0, A0 = oracle_mod.init(g.n, idx, oracle_mod.E)
        c_ref, _, _ = oracle_mod.run(g.row_ptr, g.col_ind, oracle_params(oracle_mod, ps[r]), 0, 200, X0, A0)
        np.testing.assert_array_equal(c_ens[:, r, :], c_ref, err_msg=f"replicate {r}")
    fs.fs_ens_destroy(e)
    fs.fs_graph_destroy(gh)


def test_ensemble_argument_errors(cuda):
    g = W.random_regular(1000, 4, seed=1)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    ps = scenarios(3)
    with pytest.raises(fs.FsError):
        fs.fs_ens_create(gh, scenarios(33), [1])
    mixed = scenarios(2) + scenarios(1, age_dtype=fs.FS_AGE_F16)
    with pytest.raises(fs.FsError):
        fs.fs_ens_create(gh, mixed, [1])
    e = fs.fs_ens_create(gh, ps, [1, 2])
    b = fs.fs_batch_create(fs.FS_AGE_F16, 4)
    with pytest.raises(fs.FsError):
        fs.fs_batch_add(b, e, 10)                 # age storage differs
    fs.fs_batch_destroy(b)
    b = fs.fs_batch_create(fs.FS_AGE_F32, 4)
    fs.fs_batch_add(b, e, 10)
    with pytest.raises(fs.FsError) as err:
        fs.fs_ens_destroy(e)                      # still a live member
    assert err.value.status == 5
    fs.fs_batch_run(b, 11)
    assert fs.fs_batch_status(b) == (0, 0)
    fs.fs_batch_destroy(b)
    fs.fs_ens_destroy(e)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
def test_sir_ensemble_seeded_infectious_equals_alone(cuda, pressure):
    """Index cases start in I, so the push form's initial counts come from
    them (on hub rows too): every realisation equals its run alone."""
    g = W.barabasi_albert(20_000, 5, seed=31)
    idx = W.index_nodes(g.n, 25, seed=32)          # hubs allowed
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    ps = [fs.sim_params(fs.FS_SIR, fs.law("lognormal", math.log(5.0), 0.5 + 0.05 * r), 0.1 + 0.03 * r, 0.1,
                        seed=77 + r, replicate=r, pressure=pressure) for r in range(9)]
    e = fs.fs_ens_create(gh, ps, idx)
    c_ens = fs.fs_ens_run(e, 150, 9, graph_steps=30)
    for r in range(9):
        c, X, _ = alone(gh, g.n, ps[r], idx, 150)
        np.testing.assert_array_equal(c_ens[:, r, :], c, err_msg=f"replicate {r}")
    assert c_ens[-1, :, 3].min() > 0
    fs.fs_ens_destroy(e)
    fs.fs_graph_destroy(gh)


def test_default_form_follows_replicate_width():
    """FS_PRESSURE_AUTO gives a packed ensemble the push form at up to 8
    realisations (8 replicate lanes) and the gather above; explicit flags and
    a shedding profile (gather only) decide it otherwise."""
    import torch
    assert torch.cuda.is_available()
    g = W.random_regular(4_000, 6, seed=31)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    idx = W.index_nodes(g.n, 10, seed=32)
    cases = [(scenarios(5), fs.FS_PRESSURE_PUSH), (scenarios(8), fs.FS_PRESSURE_PUSH),
             (scenarios(12), fs.FS_PRESSURE_GATHER), (scenarios(5, pressure=fs.FS_PRESSURE_GATHER), fs.FS_PRESSURE_GATHER),
             (scenarios(20, pressure=fs.FS_PRESSURE_PUSH), fs.FS_PRESSURE_PUSH)]
    shed = scenarios(3)
    for p in shed:
        p.shed_mode = fs.FS_SHED_HAZARD
        p.shedding = fs.law("exp", 1.0)
    cases.append((shed, fs.FS_PRESSURE_GATHER))
    for params, form in cases:
        e = fs.fs_ens_create(gh, params, idx)
        assert fs.fs_ens_pressure_get(e) == form, (len(params), params[0].flags, form)
        fs.fs_ens_destroy(e)
    fs.fs_graph_destroy(gh)
