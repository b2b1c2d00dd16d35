"""GPU parity of the source-node infectivity with a shedding profile
(Section 5.3, Eq. 8) against the oracle, through the C ABI.

The kernel evaluates beta s(tau') in FP32 for every node that is I after a
step, stores it in the age storage type, and sums the stored values of an S
node's infectious in-neighbours in FP32 in a fixed order. The tests check:
  - the FP32 densities (FS_SHED_DENSITY) against the oracle's FP64 ones;
  - the stored infectivity of every I node against the oracle's
    fso_infectivity of the same age: within 2e-5 relative before the storage
    cast, so equal after it or one storage unit apart at a rounding boundary;
  - lock-step trajectories: each step, the oracle is fed the GPU's state and
    the GPU's stored infectivities and the next states must agree node by
    node, except inside a near-tie band |u - p| < 1e-6 + dt e^{-lambda dt}
    d_i 2^-24 lambda_i (the FP32 sum of d_i non-negative terms is within
    d_i 2^-24 lambda_i of the exact sum); ages bit for bit where the state
    agrees;
  - a constant profile with an exact beta s reproduces the s = 1 gather run
    bit for bit on a graph whose hub row spans several merge chunks (every
    partial is folded exactly once);
  - runs are reproducible bit for bit (the summation order is fixed), CUDA
    Graph replays equal direct launches, and checkpoint / resume is exact.
Graphs up to 1.6 * 10^6 nodes run the SELL class in the shared-memory bitmap
kernel; the N = 1.7 * 10^6 case runs it in the fused grid.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import TIE, LockstepReport, ages_as_float, oracle_params

pytestmark = pytest.mark.gpu

LN5, LN6 = math.log(5.0), math.log(6.0)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fs.load()
    return torch


def sir_shed(mode, age_dtype=fs.FS_AGE_F32, seed=1, beta=0.9, shedding=None):
    inf = fs.law("lognormal", LN5, 0.5)
    return fs.sim_params(fs.FS_SIR, inf, beta, 0.1, seed, age_dtype=age_dtype, shed_mode=mode,
                         shedding=shedding if shedding is not None else fs.law("lognormal", math.log(4.0), 0.6))


def seir_shed(mode, age_dtype=fs.FS_AGE_F32, seed=11, beta=1.2):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), beta, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), age_dtype=age_dtype, shed_mode=mode,
                         shedding=fs.law("lognormal", LN6, 0.6))


def hub_graph(seed=5):
    """BA(30,011, m = 4) plus one hub joined to 12,000 other nodes: its row
    spans four 4,096-edge merge chunks."""
    g = W.barabasi_albert(30_011, 4, seed=seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    keep = rows < g.col_ind
    u, v = rows[keep], g.col_ind[keep].astype(np.int64)
    nb = set(g.col_ind[g.row_ptr[0]:g.row_ptr[1]].tolist())
    cand = W.permutation(seed + 1, g.n, 3)
    extra = np.array([c for c in cand[:13_000] if c != 0 and c not in nb][:12_000], dtype=np.int64)
    u = np.concatenate([u, np.zeros(extra.size, dtype=np.int64)])
    v = np.concatenate([v, extra])
    return W.csr_from_edges(g.n, u, v, "ba+hub")


def rho_float(rho, age_dtype):
    return ages_as_float(rho, age_dtype)


def storage_ulp(x, age_dtype):
    x = np.abs(np.asarray(x, dtype=np.float64))
    bits = {fs.FS_AGE_F32: 23, fs.FS_AGE_F16: 10, fs.FS_AGE_BF16: 7}[age_dtype]
    e = np.floor(np.log2(np.maximum(x, 1e-38)))
    return np.exp2(e - bits)


def shed_lockstep(om, g, params, sim, steps, rep):
    prm = oracle_params(om, params)
    deg = np.diff(g.row_ptr)
    for _ in range(steps):
        X, A, k = fs.fs_sim_get_state(sim, g.n, params.age_dtype)
        Af = ages_as_float(A, params.age_dtype)
        rho = rho_float(fs.fs_sim_infectivity_get(sim, g.n, params.age_dtype), params.age_dtype)
        inf_nodes = np.flatnonzero(X == fs.FS_I)
        assert (rho[X != fs.FS_I] == 0).all()
        if inf_nodes.size > 50_000:                  # a fixed sample on large graphs
            inf_nodes = inf_nodes[np.linspace(0, inf_nodes.size - 1, 50_000).astype(np.int64)]
        ref = np.array([om.infectivity(prm, float(Af[i])) for i in inf_nodes], dtype=np.float64)
        got = rho[inf_nodes].astype(np.float64)
        # relative error means nothing below the smallest normal FP32 value,
        # where the FP32 profile may flush to 0 a value the oracle rounds to a
        # subnormal
        tol = np.maximum(np.maximum(2e-5 * np.abs(ref), storage_ulp(ref, params.age_dtype) * 1.0001), 2.0 ** -126)
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (k, inf_nodes[bad][:5], got[bad][:5], ref[bad][:5])
        rep.rho_checked += inf_nodes.size
        Xo, Ao, _, margin, lam = om.step_rho(g.row_ptr, g.col_ind, prm, k, X, Af, rho_in=rho)
        fs.fs_sim_step(sim)
        X2, A2, k2 = fs.fs_sim_get_state(sim, g.n, params.age_dtype)
        assert k2 == k + 1
        band = TIE + params.dt * np.exp(-lam * params.dt) * deg * 2.0 ** -24 * lam * 1.01
        trials = np.isfinite(margin)
        rep.decisions += int(trials.sum())
        rep.node_steps += g.n
        rep.near_ties += int((np.abs(margin[trials]) < band[trials]).sum())
        mism = X2 != Xo
        if mism.any():
            assert (np.abs(margin[mism]) < band[mism]).all(), (k, np.flatnonzero(mism)[:10], margin[mism][:10])
            rep.mismatches += int(mism.sum())
        ok = ~mism
        same = ages_as_float(A2, params.age_dtype)[ok].view(np.uint32) == Ao[ok].view(np.uint32)
        assert same.all(), f"step {k}: age mismatch at {np.flatnonzero(ok)[~same][:10]}"
    assert rep.mismatches <= 1e-6 * rep.decisions, (rep.mismatches, rep.decisions)
    return rep


def test_density_fp32_against_oracle(torch_cuda, oracle_mod):
    torch = torch_cuda
    taus = np.concatenate([np.array([0.0, 1e-6, 1e-3], dtype=np.float32),
                           (np.arange(1, 3001, dtype=np.float32) * np.float32(0.02)).astype(np.float32)])
    t_dev = torch.from_numpy(taus).cuda()
    f_dev = torch.empty_like(t_dev)
    for kind, a, b, k in [("lognormal", LN5, 0.5, 0), ("lognormal", math.log(4.0), 0.668, 0),
                          ("weibull", 2.0, 4.0, 0), ("weibull", 1.5, 2.0, 0), ("erlang", 0.75, 0.0, 3),
                          ("erlang", 2.0, 0.0, 7), ("exp", 0.2, 0.0, 0)]:
        fs.fs_eval_density(fs.law(kind, a, b, k), t_dev, f_dev)
        torch.cuda.synchronize()
        f = f_dev.cpu().numpy().astype(np.float64)
        olaw = oracle_mod.law(kind, a, b, k)
        ref = np.array([oracle_mod.density(olaw, float(t)) for t in taus])
        fmax = ref.max()
        big = ref >= 1e-30 * fmax
        # the exponent's FP32 rounding grows with its magnitude |ln(f / fmax)|
        tol = 2e-6 * (5.0 + np.abs(np.log(ref[big] / fmax)))
        rel = np.abs(f[big] - ref[big]) / ref[big]
        assert (rel <= tol).all(), (kind, taus[big][np.argmax(rel / tol)], rel.max())
        assert (np.abs(f[~big]) <= 1e-29 * fmax).all()


@pytest.mark.parametrize("mode", [fs.FS_SHED_DENSITY, fs.FS_SHED_HAZARD], ids=["density", "hazard"])
@pytest.mark.parametrize("age_dtype", [fs.FS_AGE_F32, fs.FS_AGE_BF16], ids=["f32", "bf16"])
def test_sir_regular_lockstep(torch_cuda, oracle_mod, mode, age_dtype):
    """SIR on a 10-regular graph, N = 10^4 (SELL class only), 120 steps."""
    g = W.random_regular(10_000, 10, seed=0)
    idx = W.index_nodes(g.n, 30, seed=1)
    p = sir_shed(mode, age_dtype=age_dtype)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, idx)
    assert fs.fs_sim_pressure_get(s) == fs.FS_PRESSURE_GATHER
    rep = LockstepReport()
    rep.rho_checked = 0
    shed_lockstep(oracle_mod, g, p, s, 120, rep)
    c = fs.fs_sim_run(s, 1, graph_steps=1)
    assert c[-1, 3] > 100 and rep.rho_checked > 10_000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


@pytest.mark.parametrize("dispatch", [fs.FS_DISPATCH_AUTO, fs.FS_DISPATCH_MERGE], ids=["auto", "merge"])
def test_seir_hub_graph_lockstep(torch_cuda, oracle_mod, dispatch):
    """SEIR on BA + a 12,000-edge hub: merge-class rows, cross-chunk partials."""
    g = hub_graph()
    idx = W.index_nodes(g.n, 60, seed=2, allowed=W.non_hub_nodes(g))
    p = seir_shed(fs.FS_SHED_DENSITY)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(dispatch, 0))
    info = fs.fs_graph_info_get(gh)
    assert info["n_merge"] > 0 and info["merge_chunks"] >= 4
    s = fs.fs_sim_init(gh, p, idx)
    rep = LockstepReport()
    rep.rho_checked = 0
    shed_lockstep(oracle_mod, g, p, s, 40, rep)
    fs.fs_sim_run(s, 150, want_counts=False)
    shed_lockstep(oracle_mod, g, p, s, 30, rep)
    assert rep.decisions > 10_000 and rep.rho_checked > 1000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_large_graph_global_bitmap_kernel(torch_cuda, oracle_mod):
    """N = 1.7 * 10^6: the bitmap (212 KB) exceeds the shared-memory limit, so
    the SELL class runs in the fused grid; a mid-epidemic state (S 50%, I
    30% with ages up to 15 d, R 20%) set through set_state."""
    n = 1_700_000
    g = W.random_regular(n, 4, seed=21)
    rng = np.random.default_rng(5)
    X = rng.choice([fs.FS_S, fs.FS_I, fs.FS_R], n, p=[0.5, 0.3, 0.2]).astype(np.uint8)
    A = np.where(X == fs.FS_I, rng.uniform(0, 15, n), 0).astype(np.float32)
    p = sir_shed(fs.FS_SHED_DENSITY, seed=23)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, p, [0])
    fs.fs_sim_set_state(s, X, A, 7)
    rep = LockstepReport()
    rep.rho_checked = 0
    shed_lockstep(oracle_mod, g, p, s, 3, rep)
    assert rep.decisions > 1_000_000
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_constant_profile_equals_markovian_edges(torch_cuda):
    """s = hazard of Exp(2) = 2, beta = 0.125: every stored rho is 0.25 and
    every FP32 partial sum is exact, so the run equals the s = 1 gather run
    with beta = 0.25 bit for bit, whichever class holds a row."""
    g = hub_graph(seed=9)
    idx = W.index_nodes(g.n, 40, seed=3, allowed=W.non_hub_nodes(g))
    for dispatch in (fs.FS_DISPATCH_AUTO, fs.FS_DISPATCH_MERGE):
        gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(dispatch, 0))
        for age_dtype in (fs.FS_AGE_F32, fs.FS_AGE_BF16):
            lat, inf = fs.law("weibull", 2.0, 4.0), fs.law("lognormal", LN6, 0.6)
            base = fs.sim_params(fs.FS_SEIR, inf, 0.25, 0.1, 7, latent=lat, age_dtype=age_dtype,
                                 pressure=fs.FS_PRESSURE_GATHER)
            shed = fs.sim_params(fs.FS_SEIR, inf, 0.125, 0.1, 7, latent=lat, age_dtype=age_dtype,
                                 shed_mode=fs.FS_SHED_HAZARD, shedding=fs.law("exp", 2.0))
            a = fs.fs_sim_init(gh, base, idx)
            b = fs.fs_sim_init(gh, shed, idx)
            ca = fs.fs_sim_run(a, 300, graph_steps=50)
            cb = fs.fs_sim_run(b, 300, graph_steps=50)
            assert ca[-1, 3] > 1000
            np.testing.assert_array_equal(ca, cb)
            Xa, Aa, _ = fs.fs_sim_get_state(a, g.n, age_dtype)
            Xb, Ab, _ = fs.fs_sim_get_state(b, g.n, age_dtype)
            np.testing.assert_array_equal(Xa, Xb)
            np.testing.assert_array_equal(Aa.view(np.uint8), Ab.view(np.uint8))
            rho = rho_float(fs.fs_sim_infectivity_get(b, g.n, age_dtype), age_dtype)
            assert (rho[Xb == fs.FS_I] == 0.25).all() and (rho[Xb != fs.FS_I] == 0).all()
            fs.fs_sim_destroy(a)
            fs.fs_sim_destroy(b)
        fs.fs_graph_destroy(gh)


def test_reproducible_replay_and_resume(torch_cuda):
    """Two runs are identical (fixed summation order); graph replays equal
    direct launches; a checkpoint taken mid-run resumes exactly (the
    infectivity is rebuilt from the stored ages)."""
    g = hub_graph(seed=13)
    idx = W.index_nodes(g.n, 40, seed=4, allowed=W.non_hub_nodes(g))
    p = seir_shed(fs.FS_SHED_HAZARD, age_dtype=fs.FS_AGE_BF16, seed=17)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    a = fs.fs_sim_init(gh, p, idx)
    b = fs.fs_sim_init(gh, p, idx)
    ca = fs.fs_sim_run(a, 157, graph_steps=50)
    cb = np.zeros_like(ca)
    cb[0] = ca[0]
    for k in range(157):
        cb[k + 1] = fs.fs_sim_run(b, 1, graph_steps=1)[1]
    np.testing.assert_array_equal(ca, cb)
    X, A, k = fs.fs_sim_get_state(a, g.n, p.age_dtype)
    rho_a = fs.fs_sim_infectivity_get(a, g.n, p.age_dtype)
    c = fs.fs_sim_init(gh, p, idx)
    fs.fs_sim_set_state(c, X, A, k)
    np.testing.assert_array_equal(fs.fs_sim_infectivity_get(c, g.n, p.age_dtype), rho_a)
    ra = fs.fs_sim_run(a, 120, graph_steps=50)
    rc = fs.fs_sim_run(c, 120, graph_steps=50)
    np.testing.assert_array_equal(ra, rc)
    Xa, Aa, _ = fs.fs_sim_get_state(a, g.n, p.age_dtype)
    Xc, Ac, _ = fs.fs_sim_get_state(c, g.n, p.age_dtype)
    np.testing.assert_array_equal(Xa, Xc)
    np.testing.assert_array_equal(Aa, Ac)
    for s in (a, b, c):
        fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)


def test_shedding_argument_errors(torch_cuda):
    g = W.random_regular(300, 4, seed=1)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    bad = sir_shed(fs.FS_SHED_DENSITY)
    bad.shed_mode = 3
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, bad, [1])
    assert e.value.status == 1
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_init(gh, sir_shed(fs.FS_SHED_HAZARD, shedding=fs.law("none")), [1])
    assert e.value.status == 1
    for p in [sir_shed(fs.FS_SHED_DENSITY), sir_shed(fs.FS_SHED_HAZARD)]:
        p.flags = fs.FS_PRESSURE_PUSH
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_init(gh, p, [1])
        assert e.value.status == 7
    # the adaptive step combines with a profile (gather form)
    p = sir_shed(fs.FS_SHED_DENSITY)
    p.eps = 0.05
    s = fs.fs_sim_init(gh, p, [1])
    assert fs.fs_sim_pressure_get(s) == fs.FS_PRESSURE_GATHER
    fs.fs_sim_destroy(s)
    # packed ensembles take profiles in the gather form, not in the push form
    ens = fs.fs_ens_create(gh, [sir_shed(fs.FS_SHED_DENSITY, seed=k) for k in range(3)], [1])
    fs.fs_ens_destroy(ens)
    pp = [sir_shed(fs.FS_SHED_DENSITY, seed=k) for k in range(3)]
    for q in pp:
        q.flags = fs.FS_PRESSURE_PUSH
    with pytest.raises(fs.FsError) as e:
        fs.fs_ens_create(gh, pp, [1])
    assert e.value.status == 7
    s = fs.fs_sim_init(gh, fs.sim_params(fs.FS_SIR, fs.law("exp", 0.2), 0.3, 0.1, 1), [1])
    with pytest.raises(fs.FsError) as e:
        fs.fs_sim_infectivity_get(s, g.n)
    assert e.value.status == 7
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
