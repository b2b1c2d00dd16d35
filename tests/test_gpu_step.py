"""GPU parity of the fused step against the oracle, through the C ABI.

Covers: FP32 hazards within 1e-5 relative of the FP64 oracle (Section 5.1);
Philox uniforms bit-exact; lock-step trajectories on the SIR parity workload
(10-regular, N = 10^4, 300 steps) and on reduced SEIR workloads (regular and
Barabasi-Albert, several tiles plus a ragged tail); dispatch invariance
(thread / merge classes give bit-identical trajectories, Section 5.5); CUDA
Graph replay equal to direct launches (Algorithm 2); FP16/BF16 age storage
(Section 5.7); checkpoint and resume; edge cases and argument errors. Every
trajectory test runs both forms of the pressure (the gather of Algorithm 3
and the push form), which must each match the oracle; a directed graph checks
that the push form follows the transposed rows.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import LockstepReport, ages_as_float, lockstep, oracle_params

pytestmark = pytest.mark.gpu

LN5, LN6 = math.log(5.0), math.log(6.0)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fs.load()
    return torch


PRESSURES = [pytest.param(fs.FS_PRESSURE_GATHER, id="gather"), pytest.param(fs.FS_PRESSURE_PUSH, id="push")]


def c0_params(seed=1, age_dtype=fs.FS_AGE_F32, pressure=fs.FS_PRESSURE_AUTO):
    return fs.sim_params(fs.FS_SIR, fs.law("lognormal", LN5, 0.5), 0.3, 0.1, seed, age_dtype=age_dtype,
                         pressure=pressure)


def seir_params(seed=1, age_dtype=fs.FS_AGE_F32, replicate=0, pressure=fs.FS_PRESSURE_AUTO):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 0.25, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), age_dtype=age_dtype, replicate=replicate,
                         pressure=pressure)


# ----------------------------------------------------------------- primitives
LAWS = [
    ("lognormal", LN5, 0.5, 0), ("lognormal", LN6, 0.6, 0), ("lognormal", LN6, 0.3, 0),
    ("lognormal", LN6, 1.0, 0), ("lognormal", math.log(4), 0.668, 0), ("weibull", 2.0, 4.0, 0),
    ("weibull", 1.5, 2.0, 0), ("erlang", 0.75, 0.0, 3), ("erlang", 2.0, 0.0, 7), ("exp", 0.2, 0.0, 0),
]


@pytest.mark.parametrize("kind,a,b,k", LAWS)
def test_hazard_fp32_within_1e5_of_oracle(torch_cuda, oracle_mod, kind, a, b, k):
    torch = torch_cuda
    taus = np.concatenate([
        np.array([0.0, 1e-30, 1e-6, 1e-3], dtype=np.float32),
        (np.arange(1, 3001, dtype=np.float32) * np.float32(0.1)).astype(np.float32),
        np.arange(0, 1 << 15, dtype=np.uint16).view(np.float16).astype(np.float32)[:0x7800],
    ])
    taus = taus[np.isfinite(taus) & (taus >= 0)]
    t_dev = torch.from_numpy(taus).cuda()
    h_dev = torch.empty_like(t_dev)
    lw = fs.law(kind, a, b, k)
    fs.fs_eval_hazard(lw, t_dev, h_dev)
    torch.cuda.synchronize()
    h = h_dev.cpu().numpy().astype(np.float64)
    olaw = oracle_mod.law(kind, a, b, k)
    ref = np.array([oracle_mod.hazard(olaw, float(t)) for t in taus])
    big = ref >= 1e-30
    rel = np.abs(h[big] - ref[big]) / ref[big]
    assert rel.max() <= 1e-5, (taus[big][rel.argmax()], h[big][rel.argmax()], ref[big][rel.argmax()])
    assert (h[~big] <= 1e-30).all()


def test_uniforms_bit_exact(torch_cuda, oracle_mod):
    torch = torch_cuda
    rng = np.random.default_rng(0)
    for seed, rep, step in [(1, 0, 0), (1, 0, 299), (0xDEADBEEF12345678, 5, 77), (2**64 - 1, 3, 2**31)]:
        nodes = rng.integers(0, 2**31 - 1, 4096).astype(np.int32)
        nodes[:4] = [0, 1, 2, 2**31 - 2]
        nd = torch.from_numpy(nodes).cuda()
        u = torch.empty(nodes.size, dtype=torch.float32, device="cuda")
        fs.fs_eval_uniforms(seed, rep, step, nd, u)
        torch.cuda.synchronize()
        got = u.cpu().numpy().astype(np.float64)
        ref = np.array([oracle_mod.uniform(seed, rep, step, int(v)) for v in nodes])
        np.testing.assert_array_equal(got, ref)


# ----------------------------------------------------------------- trajectories
@pytest.mark.parametrize("pressure", PRESSURES)
def test_c0_sir_regular_lockstep_and_free_run(torch_cuda, oracle_mod, pressure):
    """SIR on the 10-regular parity graph, N = 10^4, 300 steps (the small workload)."""
    g = W.random_regular(10_000, 10, seed=0)
    idx = W.index_nodes(g.n, 10, seed=1)
    p = c0_params(pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    info = fs.fs_graph_info_get(gh)
    assert info["identity_layout"] == 1 and info["n_merge"] == 0 and info["d_max"] == 10
    s = fs.fs_sim_init(gh, p, idx)
    assert fs.fs_sim_pressure_get(s) == pressure
    rep = lockstep(oracle_mod, g, p, s, 300)
    assert rep.mismatches == 0
    fs.fs_sim_destroy(s)
    # the free run through captured CUDA Graphs equals the oracle's free run
    s2 = fs.fs_sim_init(gh, p, idx)
    c_gpu = fs.fs_sim_run(s2, 300, graph_steps=50)
    X0, A0 = oracle_mod.init(g.n, idx, oracle_mod.I)
    c_ref, Xr, Ar = oracle_mod.run(g.row_ptr, g.col_ind, oracle_params(oracle_mod, p), 0, 300, X0, A0)
    np.testing.assert_array_equal(c_gpu, c_ref)
    Xg, Ag, kg = fs.fs_sim_get_state(s2, g.n)
    assert kg == 300
    np.testing.assert_array_equal(Xg, Xr)
    np.testing.assert_array_equal(Ag.view(np.uint32), Ar.view(np.uint32))
    w = fs.fs_sim_work(s2)
    assert w["steps"] == 300 and w["s_node_sum"] == int(c_ref[:-1, 0].astype(np.int64).sum())
    assert w["s_degree_sum"] == 10 * w["s_node_sum"]
    fs.fs_sim_destroy(s2)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("graph_steps", [1, 7, 50, 256])
def test_graph_replay_equals_direct_launches(torch_cuda, graph_steps, pressure):
    g = W.random_regular(20_018, 8, seed=3)
    idx = W.index_nodes(g.n, 30, seed=4)
    p = seir_params(seed=9, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    sa = fs.fs_sim_init(gh, p, idx)
    sb = fs.fs_sim_init(gh, p, idx)
    ca = fs.fs_sim_run(sa, 333, graph_steps=graph_steps)
    cb = np.vstack([fs.fs_sim_run(sb, 0)] + [fs.fs_sim_step(sb)[None, :] for _ in range(333)])
    np.testing.assert_array_equal(ca, cb)
    Xa, Aa, _ = fs.fs_sim_get_state(sa, g.n)
    Xb, Ab, _ = fs.fs_sim_get_state(sb, g.n)
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(Aa.view(np.uint32), Ab.view(np.uint32))
    for s in (sa, sb):
        fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
def test_seir_regular_lockstep_reduced(torch_cuda, oracle_mod, pressure):
    """The 10-regular SEIR workload at N = 10^5 (many tiles)."""
    g = W.random_regular(100_000, 10, seed=0)
    idx = W.index_nodes(g.n, 100, seed=1)
    p = seir_params(pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    fs.fs_sim_run(s, 150, want_counts=False)       # reach the growth phase
    rep = lockstep(oracle_mod, g, p, s, 40)
    assert rep.decisions > 1000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.fixture(scope="module")
def ba_small():
    return W.barabasi_albert(50_003, 5, seed=7)


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("dispatch,t1", [(fs.FS_DISPATCH_AUTO, 0), (fs.FS_DISPATCH_MERGE, 0),
                                         (fs.FS_DISPATCH_THREAD, 0), (fs.FS_DISPATCH_AUTO, 40)])
def test_ba_lockstep_each_dispatch(torch_cuda, oracle_mod, ba_small, dispatch, t1, pressure):
    g = ba_small
    idx = W.index_nodes(g.n, 50, seed=2, allowed=W.non_hub_nodes(g))
    p = seir_params(seed=11, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(dispatch, t1))
    info = fs.fs_graph_info_get(gh)
    if dispatch != fs.FS_DISPATCH_THREAD:
        assert info["n_merge"] > 0 and info["merge_chunks"] > 0 and info["identity_layout"] == 0
    if pressure == fs.FS_PRESSURE_PUSH and info["thread_max_deg"] > 255:
        # every node in the one-thread-per-node class: u8 counts cannot hold its in-degrees
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_init(gh, p, idx)
        assert e.value.status == 7
        fs.fs_graph_destroy(gh)
        return
    s = fs.fs_sim_init(gh, p, idx)
    assert fs.fs_sim_pressure_get(s) == pressure
    rep = LockstepReport()
    lockstep(oracle_mod, g, p, s, 25, rep)
    fs.fs_sim_run(s, 60, want_counts=False)
    lockstep(oracle_mod, g, p, s, 25, rep)
    assert rep.decisions > 1000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_dispatch_classes_bit_identical(torch_cuda, ba_small):
    """Integer pressure makes every traversal class and both pressure forms
    exact: the same trajectory."""
    g = ba_small
    idx = W.index_nodes(g.n, 50, seed=2, allowed=W.non_hub_nodes(g))
    results = []
    for dispatch, t1, pressure in [(fs.FS_DISPATCH_AUTO, 0, fs.FS_PRESSURE_GATHER),
                                   (fs.FS_DISPATCH_MERGE, 0, fs.FS_PRESSURE_GATHER),
                                   (fs.FS_DISPATCH_THREAD, 0, fs.FS_PRESSURE_GATHER),
                                   (fs.FS_DISPATCH_AUTO, 100, fs.FS_PRESSURE_GATHER),
                                   (fs.FS_DISPATCH_AUTO, 255, fs.FS_PRESSURE_GATHER),
                                   (fs.FS_DISPATCH_AUTO, 0, fs.FS_PRESSURE_PUSH),
                                   (fs.FS_DISPATCH_MERGE, 0, fs.FS_PRESSURE_PUSH),
                                   (fs.FS_DISPATCH_AUTO, 255, fs.FS_PRESSURE_PUSH),
                                   (fs.FS_DISPATCH_THREAD, 0, fs.FS_PRESSURE_AUTO)]:
        p = seir_params(seed=5, pressure=pressure)
        gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(dispatch, t1))
        s = fs.fs_sim_init(gh, p, idx)
        if dispatch == fs.FS_DISPATCH_THREAD:
            # d_max > 255 in the thread class: AUTO falls back to the gather
            assert fs.fs_sim_pressure_get(s) == fs.FS_PRESSURE_GATHER
        c = fs.fs_sim_run(s, 400)
        X, A, _ = fs.fs_sim_get_state(s, g.n)
        results.append((c, X, A))
        fs.fs_sim_destroy(s)
        fs.fs_graph_destroy(gh)
    for c, X, A in results[1:]:
        np.testing.assert_array_equal(c, results[0][0])
        np.testing.assert_array_equal(X, results[0][1])
        np.testing.assert_array_equal(A.view(np.uint32), results[0][2].view(np.uint32))
    assert results[0][0][-1, 3] > 0


@pytest.mark.parametrize("pressure", PRESSURES)
@pytest.mark.parametrize("age_dtype", [fs.FS_AGE_F16, fs.FS_AGE_BF16])
def test_reduced_precision_ages_lockstep(torch_cuda, oracle_mod, age_dtype, pressure):
    g = W.erdos_renyi(30_001, 8, seed=2)
    idx = W.index_nodes(g.n, 60, seed=3)
    p = seir_params(seed=21, age_dtype=age_dtype, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    rep = LockstepReport()
    lockstep(oracle_mod, g, p, s, 20, rep)
    fs.fs_sim_run(s, 300, want_counts=False)       # ages beyond 32 d freeze in bf16
    lockstep(oracle_mod, g, p, s, 20, rep)
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("pressure", PRESSURES)
def test_checkpoint_resume_is_exact(torch_cuda, ba_small, pressure):
    g = ba_small
    idx = W.index_nodes(g.n, 40, seed=9, allowed=W.non_hub_nodes(g))
    p = seir_params(seed=33, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    c_all = fs.fs_sim_run(s, 300)
    X_all, A_all, _ = fs.fs_sim_get_state(s, g.n)
    fs.fs_sim_destroy(s)
    s = fs.fs_sim_init(gh, p, idx)
    c1 = fs.fs_sim_run(s, 120)
    X, A, k = fs.fs_sim_get_state(s, g.n)
    fs.fs_sim_destroy(s)
    s = fs.fs_sim_init(gh, p, [])
    fs.fs_sim_set_state(s, X, A, k)
    c2 = fs.fs_sim_run(s, 180)
    X2, A2, k2 = fs.fs_sim_get_state(s, g.n)
    assert k2 == 300
    np.testing.assert_array_equal(np.vstack([c1, c2[1:]]), c_all)
    np.testing.assert_array_equal(X2, X_all)
    np.testing.assert_array_equal(A2.view(np.uint32), A_all.view(np.uint32))
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def directed_graph(n: int, m: int, seed: int):
    """A directed graph with skewed in- and out-degrees: rows list in-neighbours;
    node j's out-neighbours are the rows that list j (not its own row)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = (rng.pareto(1.5, m) * 3).astype(np.int64) % n          # skewed in-degrees
    src = np.concatenate([src, np.arange(n)])                      # a directed ring
    dst = np.concatenate([dst, (np.arange(n) + 1) % n])
    keep = src != dst                                              # simple: no loops, no repeats
    pairs = np.unique(np.stack([dst[keep], src[keep]], axis=1), axis=0)
    dst, src = pairs[:, 0], pairs[:, 1]
    order = np.argsort(dst, kind="stable")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, dst + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return W.Graph(n, row_ptr, src[order].astype(np.int32), "directed")


@pytest.mark.parametrize("pressure", PRESSURES)
def test_directed_graph_free_run(torch_cuda, oracle_mod, pressure):
    """On a directed graph the pressure counts in-neighbours (rows), so the
    push form must push along the transposed rows; both forms match the oracle."""
    g = directed_graph(20_000, 150_000, seed=4)
    assert not np.array_equal(np.sort(g.col_ind), np.sort(np.repeat(np.arange(g.n), np.diff(g.row_ptr))))
    idx = W.index_nodes(g.n, 40, seed=5)
    p = seir_params(seed=17, pressure=pressure)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    c = fs.fs_sim_run(s, 400)
    X0, A0 = oracle_mod.init(g.n, idx, oracle_mod.E)
    c_ref, Xr, Ar = oracle_mod.run(g.row_ptr, g.col_ind, oracle_params(oracle_mod, p), 0, 400, X0, A0)
    np.testing.assert_array_equal(c, c_ref)
    Xg, Ag, _ = fs.fs_sim_get_state(s, g.n)
    np.testing.assert_array_equal(Xg, Xr)
    np.testing.assert_array_equal(Ag.view(np.uint32), Ar.view(np.uint32))
    assert c_ref[-1, 3] > 100
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


# ----------------------------------------------------------------- edge cases
@pytest.mark.parametrize("pressure", PRESSURES)
def test_edge_cases_tiny_and_ragged(torch_cuda, oracle_mod, pressure):
    # one node, no edges; every node infectious; nothing infectious; ragged sizes
    for n, edges, idx, steps in [(1, None, [0], 50), (33, None, list(range(33)), 80),
                                 (1000, "ring", [], 20), (65, "ring", [64], 120), (4097, "ring", [0, 4096], 200)]:
        if edges is None:
            g = W.empty_graph(n)
        else:
            u = np.arange(n, dtype=np.int64)
            g = W.csr_from_edges(n, u, (u + 1) % n)
        p = c0_params(seed=n, pressure=pressure)
        gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
        s = fs.fs_sim_init(gh, p, np.array(idx, dtype=np.int32))
        c = fs.fs_sim_run(s, steps)
        X0, A0 = oracle_mod.init(n, np.array(idx, dtype=np.int32), oracle_mod.I)
        c_ref, Xr, Ar = oracle_mod.run(g.row_ptr, g.col_ind, oracle_params(oracle_mod, p), 0, steps, X0, A0)
        np.testing.assert_array_equal(c, c_ref)
        fs.fs_sim_destroy(s)
        fs.fs_graph_destroy(gh)


def test_argument_errors(torch_cuda):
    g = W.random_regular(100, 4, seed=1)
    with pytest.raises(fs.FsError) as e:
        bad = g.row_ptr.copy()
        bad[5] = bad[6] + 1
        fs.fs_graph_create(g.n, bad, g.col_ind)
    assert e.value.status == 1
    with pytest.raises(fs.FsError) as e:
        badc = g.col_ind.copy()
        badc[3] = 100
        fs.fs_graph_create(g.n, g.row_ptr, badc)
    assert e.value.status == 1
    with pytest.raises(fs.FsError) as e:
        fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, weights=np.ones(g.nnz, dtype=np.float32))
    assert e.value.status == 7
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    for bad_p in [fs.sim_params(fs.FS_SIR, fs.law("lognormal", 1.0, -1.0), 0.3, 0.1, 1),
                  fs.sim_params(fs.FS_SIR, fs.law("lognormal", 1.0, 0.5), 0.3, 0.0, 1),
                  fs.sim_params(fs.FS_SEIR, fs.law("exp", 0.1), 0.3, 0.1, 1),
                  fs.sim_params(fs.FS_SIR, fs.law("exp", 0.1), 0.3, 0.1, 1, index_state=fs.FS_E)]:
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_init(gh, bad_p, [1, 2])
        assert e.value.status == 1
    p = c0_params()
    with pytest.raises(fs.FsError):
        fs.fs_sim_init(gh, p, [1, 1])
    with pytest.raises(fs.FsError):
        fs.fs_sim_init(gh, p, [100])
    s = fs.fs_sim_init(gh, p, [1])
    with pytest.raises(fs.FsError) as e:
        fs.fs_graph_destroy(gh)
    assert e.value.status == 5
    X, A, k = fs.fs_sim_get_state(s, g.n)
    A[0] = 1.0                       # S node with a non-zero age
    with pytest.raises(fs.FsError):
        fs.fs_sim_set_state(s, X, A, k)
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
