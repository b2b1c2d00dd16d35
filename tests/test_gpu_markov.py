"""GPU parity of the Markovian engine (Section 4, Algorithm 1) against the
oracle, through the C ABI.

Lock-step: each step the oracle takes the GPU's state, computes Algorithm 1's
step size from it (in double from integer reductions, as the kernels do: the
two must agree bit for bit, which the next state and the simulated clock
check) and one step of that size; the GPU's next state must agree node by
node outside the Bernoulli near-tie band, ages bit for bit where the state
agrees, and the clock must equal the FP64 sum of the oracle's step sizes.
Inertial and Control modes (event pushes vs dense recount) give identical
runs; graph replays equal direct launches; argument errors.
"""
import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import TIE, ages_as_float, oracle_params

pytestmark = pytest.mark.gpu

THETA, PMAX = 0.01, 0.1


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fs.load()
    return torch


def mk_params(model, seed=3, mode=0, age_dtype=fs.FS_AGE_F32):
    lat = fs.law("exp", 0.3) if model == fs.FS_SEIR else None
    return fs.sim_params(model, fs.law("exp", 0.15), 0.25, 0.1, seed, latent=lat, age_dtype=age_dtype,
                         theta=THETA, p_max=PMAX, markov_mode=mode)


def markov_lockstep(om, g, p, sim, steps):
    prm = oracle_params(om, p)
    t0, _ = fs.fs_sim_time(sim)
    taus = []
    mism = decisions = 0
    for _ in range(steps):
        X, A, k = fs.fs_sim_get_state(sim, g.n, p.age_dtype)
        Af = ages_as_float(A, p.age_dtype)
        tau, _, _ = om.markov_tau(g.row_ptr, g.col_ind, prm, THETA, PMAX, p.dt, X)
        Xo, Ao, margin, used = om.markov_step(g.row_ptr, g.col_ind, prm, THETA, PMAX, p.dt, k, X, Af, tau_in=tau)
        assert used == tau
        fs.fs_sim_step(sim)
        X2, A2, k2 = fs.fs_sim_get_state(sim, g.n, p.age_dtype)
        assert k2 == k + 1
        bad = X2 != Xo
        trials = np.isfinite(margin)
        decisions += int(trials.sum())
        if bad.any():
            assert (np.abs(margin[bad]) < TIE).all(), (k, np.flatnonzero(bad)[:10], margin[bad][:10])
            mism += int(bad.sum())
        ok = ~bad
        same = ages_as_float(A2, p.age_dtype)[ok].view(np.uint32) == Ao[ok].view(np.uint32)
        assert same.all(), f"step {k}: age mismatch at {np.flatnonzero(ok)[~same][:10]}"
        taus.append(tau)
    assert mism <= 1e-6 * decisions, (mism, decisions)
    t = t0
    for tau in taus:
        t += float(tau)
    assert fs.fs_sim_time(sim)[0] == t
    return np.array(taus, dtype=np.float32), decisions


@pytest.mark.parametrize("model", [fs.FS_SIS, fs.FS_SIR, fs.FS_SEIR], ids=["sis", "sir", "seir"])
def test_markov_lockstep(torch_cuda, oracle_mod, model):
    g = W.erdos_renyi(20_000, 8, seed=5)
    idx = W.index_nodes(g.n, 20, seed=6)
    p = mk_params(model)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    taus, dec = markov_lockstep(oracle_mod, g, p, s, 60)
    fs.fs_sim_run(s, 300, graph_steps=50, want_counts=False)
    taus2, dec2 = markov_lockstep(oracle_mod, g, p, s, 40)
    assert dec + dec2 > 100_000
    # the theta or p_max term of Algorithm 1 binds (SEIR: only once the index
    # nodes' latent phase is over, so in the second window, steps 360-400,
    # where the oracle's own run takes tau down to 1/15)
    binding = taus2 if model == fs.FS_SEIR else taus
    assert binding.min() < p.dt
    X, _, _ = fs.fs_sim_get_state(s, g.n)
    if model == fs.FS_SIS:
        assert not (X == fs.FS_R).any() and (X == fs.FS_I).sum() > 1000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_large_graph_from_set_state(torch_cuda, oracle_mod):
    """N = 1.7 * 10^6, a mid-epidemic SIS state: every kernel strides over
    several grid rounds."""
    n = 1_700_000
    g = W.erdos_renyi(n, 6, seed=7)
    rng = np.random.default_rng(3)
    X = rng.choice([fs.FS_S, fs.FS_I], n, p=[0.7, 0.3]).astype(np.uint8)
    A = np.where(X == fs.FS_I, rng.uniform(0, 10, n), 0).astype(np.float32)
    p = mk_params(fs.FS_SIS, seed=11)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, [0])
    fs.fs_sim_set_state(s, X, A, 5)
    _, dec = markov_lockstep(oracle_mod, g, p, s, 3)
    assert dec > 3_000_000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_inertial_and_control_modes_agree(torch_cuda):
    """Barabasi-Albert (merge-class hubs in the recount): pushes of the
    events and dense recounts give the same integer counts, so the runs are
    identical; graph replays equal single-step launches."""
    g = W.barabasi_albert(50_003, 4, seed=9)
    idx = W.index_nodes(g.n, 30, seed=2, allowed=W.non_hub_nodes(g))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    info = fs.fs_graph_info_get(gh)
    assert info["n_merge"] > 0
    runs = []
    for mode in (0, 1, 2):
        s = fs.fs_sim_init(gh, mk_params(fs.FS_SIS, seed=21, mode=mode), idx)
        c = fs.fs_sim_run(s, 400, graph_steps=50)
        X, A, _ = fs.fs_sim_get_state(s, g.n)
        runs.append((c, X, A, fs.fs_sim_time(s)[0]))
        fs.fs_sim_destroy(s)
    s = fs.fs_sim_init(gh, mk_params(fs.FS_SIS, seed=21, mode=0), idx)
    c1 = np.zeros_like(runs[0][0])
    c1[0] = runs[0][0][0]
    for k in range(400):
        c1[k + 1] = fs.fs_sim_run(s, 1, graph_steps=1)[1]
    X, A, _ = fs.fs_sim_get_state(s, g.n)
    runs.append((c1, X, A, fs.fs_sim_time(s)[0]))
    fs.fs_sim_destroy(s)
    for c, X, A, t in runs[1:]:
        np.testing.assert_array_equal(c, runs[0][0])
        np.testing.assert_array_equal(X, runs[0][1])
        np.testing.assert_array_equal(A.view(np.uint32), runs[0][2].view(np.uint32))
        assert t == runs[0][3]
    assert runs[0][0][-1, 2] > 1000 and (runs[0][0][:, 3] == 0).all()
    fs.fs_graph_destroy(gh)


def test_markov_argument_errors(torch_cuda):
    g = W.random_regular(300, 4, seed=1)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    sis_fixed = fs.sim_params(fs.FS_SIS, fs.law("exp", 0.2), 0.3, 0.1, 1)
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, sis_fixed, [1])
    assert e.value.status == 7
    bad = fs.sim_params(fs.FS_SIR, fs.law("lognormal", 1.0, 0.5), 0.3, 0.1, 1, theta=0.01)
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, bad, [1])
    assert e.value.status == 1
    for kw in (dict(p_max=1.5), dict(markov_mode=3), dict(theta=float("nan"))):
        args = dict(theta=0.01)
        args.update(kw)
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_init(gh, fs.sim_params(fs.FS_SIR, fs.law("exp", 0.2), 0.3, 0.1, 1, **args), [1])
        assert e.value.status == 1
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, fs.sim_params(fs.FS_SIR, fs.law("exp", 0.2), 0.3, 0.1, 1, theta=0.01, eps=0.1), [1])
    assert e.value.status == 7
    with pytest.raises(fs.FsError) as e:
        fs.fs_ens_create(gh, [mk_params(fs.FS_SIR, seed=k) for k in range(3)], [1])
    assert e.value.status == 7
    s = fs.fs_sim_init(gh, mk_params(fs.FS_SIS), [1])
    X = np.zeros(g.n, dtype=np.uint8)
    X[3] = fs.FS_R
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_set_state(s, X, np.zeros(g.n, dtype=np.float32), 0)
    assert e.value.status == 1
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
