"""GPU parity of the adaptive step (Section 5.2) against the oracle.

Step k advances by dt_k = min(dt_max, eps / (lambda*_{k-1} + delta)), where
lambda*_{k-1} is the largest per-node rate of the previous step (beta c_i for
S nodes, the latent or infectious hazard for E/I) and the first step takes
dt_max. The GPU computes the rates, their maximum and dt_k in FP32; the oracle
in FP64. Each test checks:
  - the GPU's dt_k against the oracle's rule applied to the oracle's own
    lambda* of the GPU's previous state (relative 2e-5: the FP32 hazards are
    within 1e-5 of the oracle's, plus two roundings);
  - the GPU's next state against one oracle step of exactly the GPU's dt_k
    (lock-step; mismatches only inside the Bernoulli near-tie band), and the
    ages bit for bit wherever the state agrees;
  - the simulated clock (the FP64 sum of the step sizes).
A tolerance eps that never binds gives the fixed-step trajectory bit for bit.
Both pressure forms run the rule (the push kernel and the gather kernels'
adaptive instances), also with an age-dependent infectivity.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import TIE, LockstepReport, ages_as_float, oracle_params

pytestmark = pytest.mark.gpu

LN5, LN6 = math.log(5.0), math.log(6.0)
DT_REL = 2e-5
UNKNOWN = object()


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fs.load()
    return torch


def sir(eps, delta=0.0, age_dtype=fs.FS_AGE_F32, seed=1, pressure=fs.FS_PRESSURE_PUSH):
    return fs.sim_params(fs.FS_SIR, fs.law("lognormal", LN5, 0.5), 0.3, 0.1, seed, age_dtype=age_dtype,
                         pressure=pressure, eps=eps, delta=delta)


def seir(eps, delta=0.0, age_dtype=fs.FS_AGE_F32, seed=11, pressure=fs.FS_PRESSURE_PUSH):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 0.25, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), age_dtype=age_dtype,
                         pressure=pressure, eps=eps, delta=delta)


def adaptive_lockstep(om, g, params, sim, steps, lam_prev, rep):
    """Advance `sim` by `steps` single adaptive steps, each checked against
    the oracle; lam_prev: the oracle's lambda* of the step before the first
    (None: the first step of the run, dt = dt_max; UNKNOWN: the state came
    from a free run, so the first step's size is not checked).
    Returns (dts, lam_prev)."""
    prm = oracle_params(om, params)
    X, A, k = fs.fs_sim_get_state(sim, g.n, params.age_dtype)
    dts = []
    for _ in range(steps):
        _, dt_gpu = fs.fs_sim_time(sim)
        if lam_prev is None:
            assert dt_gpu == np.float32(params.dt)
        elif lam_prev is UNKNOWN:
            assert 0 < dt_gpu <= np.float32(params.dt)
        else:
            dt_ref = om.adaptive_dt(params.dt, params.eps, params.delta if params.delta > 0 else 1e-12, lam_prev)
            assert abs(dt_gpu - dt_ref) <= DT_REL * dt_ref, (k, dt_gpu, dt_ref, lam_prev)
        prm.dt = float(dt_gpu)
        Af = ages_as_float(A, params.age_dtype)
        Xo, Ao, margin, lam = om.step(g.row_ptr, g.col_ind, prm, k, X, Af, want_margin=True, want_lambda=True)
        fs.fs_sim_step(sim)
        X2, A2, k2 = fs.fs_sim_get_state(sim, g.n, params.age_dtype)
        assert k2 == k + 1
        bad = X2 != Xo
        trials = np.isfinite(margin)
        rep.decisions += int(trials.sum())
        rep.node_steps += g.n
        rep.near_ties += int((np.abs(margin[trials]) < TIE).sum())
        if bad.any():
            assert (np.abs(margin[bad]) < TIE).all(), (
                f"step {k}: {int(bad.sum())} state mismatches outside the tie band; margins {margin[bad][:10]}")
            rep.mismatches += int(bad.sum())
        ok = ~bad
        same = ages_as_float(A2, params.age_dtype)[ok].view(np.uint32) == Ao[ok].view(np.uint32)
        assert same.all(), f"step {k}: age mismatch at nodes {np.flatnonzero(ok)[~same][:10]}"
        dts.append(dt_gpu)
        lam_prev = float(lam.max()) if lam.size else 0.0
        X, A, k = X2, A2, k2
    assert rep.mismatches <= 1e-6 * rep.decisions, (rep.mismatches, rep.decisions)
    return np.array(dts, dtype=np.float32), lam_prev


def fp64_sum(dts):
    t = 0.0
    for d in dts:
        t += float(d)
    return t


PRESSURES = [pytest.param(fs.FS_PRESSURE_PUSH, id="push"), pytest.param(fs.FS_PRESSURE_GATHER, id="gather")]


@pytest.mark.parametrize("pressure", PRESSURES)
def test_sir_regular_adaptive_lockstep(torch_cuda, oracle_mod, pressure):
    """SIR on the 10-regular graph (N = 10^4): eps = 0.05 binds once the
    pressure builds up (beta c up to 3 per day), so dt_k drops below dt_max."""
    g = W.random_regular(10_000, 10, seed=0)
    idx = W.index_nodes(g.n, 10, seed=1)
    p = sir(0.05, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    assert fs.fs_sim_pressure_get(s) == pressure
    assert fs.fs_sim_time(s) == (0.0, np.float32(0.1))
    rep = LockstepReport()
    dts, lam = adaptive_lockstep(oracle_mod, g, p, s, 150, None, rep)
    assert rep.mismatches == 0
    assert dts.min() < 0.5 * p.dt and dts[0] == np.float32(p.dt)
    t, _ = fs.fs_sim_time(s)
    assert t == fp64_sum(dts)
    # a free run through captured CUDA Graphs, then lock-step again
    fs.fs_sim_run(s, 120, graph_steps=50, want_counts=False)
    adaptive_lockstep(oracle_mod, g, p, s, 20, UNKNOWN, rep)
    assert rep.mismatches == 0
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_free_run_equals_single_steps(torch_cuda):
    """CUDA Graph replays of the adaptive step give the trajectory, the step
    sizes and the clock of direct single-step launches, bit for bit."""
    g = W.random_regular(20_000, 8, seed=3)
    idx = W.index_nodes(g.n, 20, seed=4)
    p = sir(0.03, seed=5)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    a = fs.fs_sim_init(gh, p, idx)
    b = fs.fs_sim_init(gh, p, idx)
    ca = fs.fs_sim_run(a, 173, graph_steps=50)
    cb = np.zeros_like(ca)
    cb[0] = ca[0]
    for k in range(173):
        cb[k + 1] = fs.fs_sim_run(b, 1, graph_steps=1)[1]
    np.testing.assert_array_equal(ca, cb)
    Xa, Aa, ka = fs.fs_sim_get_state(a, g.n)
    Xb, Ab, kb = fs.fs_sim_get_state(b, g.n)
    assert ka == kb == 173
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(Aa.view(np.uint32), Ab.view(np.uint32))
    assert fs.fs_sim_time(a) == fs.fs_sim_time(b)
    assert fs.fs_sim_time(a)[0] < 173 * 0.1
    for s in (a, b):
        fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("age_dtype", [fs.FS_AGE_F32, fs.FS_AGE_BF16])
def test_seir_ba_adaptive_lockstep(torch_cuda, oracle_mod, age_dtype, pressure):
    """SEIR on a Barabasi-Albert graph (N = 50,003, m = 5): merge-class hubs
    take the per-node path; BF16 ages advance by the variable step and round
    to storage like the oracle's."""
    g = W.barabasi_albert(50_003, 5, seed=7)
    idx = W.index_nodes(g.n, 50, seed=2, allowed=W.non_hub_nodes(g))
    p = seir(0.02, delta=1e-3, age_dtype=age_dtype, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(fs.FS_DISPATCH_AUTO, 40))
    info = fs.fs_graph_info_get(gh)
    assert info["n_merge"] > 0
    s = fs.fs_sim_init(gh, p, idx)
    rep = LockstepReport()
    dts, _ = adaptive_lockstep(oracle_mod, g, p, s, 60, None, rep)
    assert rep.decisions > 1000
    assert dts.min() < p.dt
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
def test_unbinding_eps_equals_fixed_step(torch_cuda, pressure):
    """With eps / (lambda* + delta) above dt_max at every step, dt_k = dt_max
    and the adaptive kernel (direct rate evaluation) reproduces the fixed-step
    kernel (tabulated probabilities) bit for bit: the tables hold the same
    FP32 expressions."""
    g = W.barabasi_albert(30_011, 4, seed=9)
    idx = W.index_nodes(g.n, 30, seed=3, allowed=W.non_hub_nodes(g))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(fs.FS_DISPATCH_AUTO, 40))
    for mk in (lambda e: sir(e, seed=21, pressure=pressure), lambda e: seir(e, seed=22, pressure=pressure)):
        pa, pf = mk(1e6), mk(0.0)
        a = fs.fs_sim_init(gh, pa, idx)
        f = fs.fs_sim_init(gh, pf, idx)
        ca = fs.fs_sim_run(a, 200, graph_steps=50)
        cf = fs.fs_sim_run(f, 200, graph_steps=50)
        np.testing.assert_array_equal(ca, cf)
        Xa, Aa, _ = fs.fs_sim_get_state(a, g.n)
        Xf, Af, _ = fs.fs_sim_get_state(f, g.n)
        np.testing.assert_array_equal(Xa, Xf)
        np.testing.assert_array_equal(Aa.view(np.uint32), Af.view(np.uint32))
        ta, da = fs.fs_sim_time(a)
        tf, df = fs.fs_sim_time(f)
        assert da == df == np.float32(pa.dt)
        assert ta == tf == fp64_sum([np.float32(pa.dt)] * 200)
        fs.fs_sim_destroy(a)
        fs.fs_sim_destroy(f)
    fs.fs_graph_destroy(gh)


def test_set_state_restarts_step_rule(torch_cuda):
    """set_state restarts the clock and the step rule: the first step after
    it takes dt_max, as at init."""
    g = W.random_regular(5_000, 6, seed=2)
    idx = W.index_nodes(g.n, 10, seed=2)
    p = sir(0.02, seed=8)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    fs.fs_sim_run(s, 80, want_counts=False)
    t, dt = fs.fs_sim_time(s)
    assert t > 0 and dt < p.dt
    X, A, k = fs.fs_sim_get_state(s, g.n)
    fs.fs_sim_set_state(s, X, A, k)
    assert fs.fs_sim_time(s) == (0.0, np.float32(p.dt))
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_adaptive_argument_errors(torch_cuda):
    g = W.random_regular(200, 4, seed=1)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    for bad in [sir(-0.1), sir(0.05, delta=-1.0), sir(float("nan")), sir(0.05, delta=float("inf"))]:
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_init(gh, bad, [1, 2])
        assert e.value.status == 1
    # a packed ensemble takes the adaptive step in every realisation or in none
    with pytest.raises(fs.FsError) as e:
        fs.fs_ens_create(gh, [sir(0.05 if k else 0.0, seed=k) for k in range(4)], [1, 2])
    assert e.value.status == 1
    fs.fs_ens_destroy(fs.fs_ens_create(gh, [sir(0.05, seed=k) for k in range(4)], [1, 2]))
    # a fixed-step sim reports dt and the FP64 sum of its steps
    s = fs.fs_sim_init(gh, sir(0.0), [1, 2])
    fs.fs_sim_run(s, 7, want_counts=False)
    t, dt = fs.fs_sim_time(s)
    assert dt == np.float32(0.1) and t == fp64_sum([np.float32(0.1)] * 7)
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("graph", ["regular", "hub"])
def test_adaptive_with_shedding_lockstep(torch_cuda, oracle_mod, graph):
    """The paper's default renewal configuration: the adaptive step with an
    age-dependent infectivity (gather form). Each step: dt_k against the
    oracle's rule on its own lambda* (the S rates are the stored-rho sums),
    then one oracle step of the GPU's dt_k fed the GPU's stored rho."""
    from tests.test_gpu_shedding import hub_graph, rho_float
    if graph == "regular":
        g = W.random_regular(10_000, 10, seed=0)
        idx = W.index_nodes(g.n, 30, seed=1)
    else:
        g = hub_graph(seed=17)
        idx = W.index_nodes(g.n, 60, seed=2, allowed=W.non_hub_nodes(g))
    p = fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 1.2, 0.1, 31, latent=fs.law("weibull", 2.0, 4.0),
                      eps=0.03, shed_mode=fs.FS_SHED_DENSITY, shedding=fs.law("lognormal", LN6, 0.6))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    assert fs.fs_sim_pressure_get(s) == fs.FS_PRESSURE_GATHER
    om = oracle_mod
    prm = oracle_params(om, p)
    deg = np.diff(g.row_ptr)
    lam_prev = None
    dts = []
    decisions = mism = 0
    for _ in range(70):
        X, A, k = fs.fs_sim_get_state(s, g.n)
        rho = rho_float(fs.fs_sim_infectivity_get(s, g.n), fs.FS_AGE_F32)
        _, dt_gpu = fs.fs_sim_time(s)
        if lam_prev is None:
            assert dt_gpu == np.float32(p.dt)
        else:
            dt_ref = om.adaptive_dt(p.dt, p.eps, 1e-12, lam_prev)
            assert abs(dt_gpu - dt_ref) <= DT_REL * dt_ref, (k, dt_gpu, dt_ref)
        prm.dt = float(dt_gpu)
        Xo, Ao, _, margin, lam = om.step_rho(g.row_ptr, g.col_ind, prm, k, X, A, rho_in=rho)
        fs.fs_sim_step(s)
        X2, A2, _ = fs.fs_sim_get_state(s, g.n)
        band = TIE + prm.dt * np.exp(-lam * prm.dt) * deg * 2.0 ** -24 * lam * 1.01
        bad = X2 != Xo
        decisions += int(np.isfinite(margin).sum())
        if bad.any():
            assert (np.abs(margin[bad]) < band[bad]).all(), (k, np.flatnonzero(bad)[:10])
            mism += int(bad.sum())
        ok = ~bad
        assert (A2[ok].view(np.uint32) == Ao[ok].view(np.uint32)).all(), k
        dts.append(dt_gpu)
        lam_prev = float(lam.max())
    assert mism <= 1e-6 * decisions and decisions > 10_000
    assert min(dts) < p.dt
    assert fs.fs_sim_time(s)[0] == fp64_sum(dts)
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
