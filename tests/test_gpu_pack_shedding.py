"""Age-dependent shedding (Section 5.3, Eq. 8) inside packed ensembles and the
server.

Each replicate of an ensemble keeps its own infectivity beta s(tau') for the
replicates that are I, stored like the ages, and an S replicate's pressure is
the FP32 sum of the stored infectivities of its infectious in-neighbours in
the order the single-realisation gather uses (row order in the SELL class;
in the merge class the 32-edge windows, warp ranges and chunks of the merge
kernel). So every packed replicate must reproduce, bit for bit, the run it
has alone through fs_sim_* -- counts every step, final states and ages --
on a graph whose hub row spans four merge chunks, at FP32 and BF16 storage,
with two replicate widths (R_pad 8 and 16) and with the adaptive step; and
single packed steps must agree with the oracle's (lock-step, each replicate
fed to the oracle from the ensemble's state, mismatches only inside the
near-tie band that the FP32 infectivities and sums allow, ages bit for bit
where the states agree). A served request with a shedding profile equals its
realisations alone.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from paper_2604_22092_gb300._abi import FS_EINVAL, FS_EUNSUPPORTED
from tests.gpu_helpers import TIE, ages_as_float, oracle_params
from tests.test_gpu_shedding import hub_graph

pytestmark = pytest.mark.gpu

LN5, LN6 = math.log(5.0), math.log(6.0)


def shed_seir(beta, seed, replicate=0, mode=fs.FS_SHED_HAZARD, sigma=0.6, age_dtype=fs.FS_AGE_F32, eps=0.0):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, sigma), beta, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), replicate=replicate, age_dtype=age_dtype,
                         pressure=fs.FS_PRESSURE_GATHER, shed_mode=mode, eps=eps,
                         shedding=fs.law("lognormal", LN6, sigma) if mode == fs.FS_SHED_HAZARD
                         else fs.law("lognormal", math.log(4.0), 0.5))


def shed_sir(beta, seed, replicate=0, mode=fs.FS_SHED_DENSITY, age_dtype=fs.FS_AGE_F32):
    return fs.sim_params(fs.FS_SIR, fs.law("lognormal", LN5, 0.5), beta, 0.1, seed, replicate=replicate,
                         age_dtype=age_dtype, pressure=fs.FS_PRESSURE_GATHER, shed_mode=mode,
                         shedding=fs.law("lognormal", math.log(4.0), 0.6) if mode == fs.FS_SHED_DENSITY
                         else fs.law("lognormal", LN5, 0.5))


def realisations(n_real, age_dtype=fs.FS_AGE_F32, eps=0.0):
    """Quads of replicates sharing a key (one Philox call serves a quad in the
    packed step) and realisations with keys of their own; both shedding modes."""
    out = []
    for r in range(n_real):
        mode = fs.FS_SHED_HAZARD if r % 2 == 0 else fs.FS_SHED_DENSITY
        if r < n_real // 2:
            out.append(shed_seir(0.9 + 0.1 * r, seed=41, replicate=r, mode=mode, age_dtype=age_dtype, eps=eps))
        else:
            out.append(shed_seir(0.7 + 0.15 * (r % 4), seed=500 + r, mode=mode, sigma=0.4 + 0.1 * (r % 4),
                                 age_dtype=age_dtype, eps=eps))
    return out


@pytest.fixture(scope="module")
def hub():
    import torch
    assert torch.cuda.is_available()
    g = hub_graph()
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    info = fs.fs_graph_info_get(gh)
    assert info["n_merge"] > 0
    idx = W.index_nodes(g.n, 40, seed=3, allowed=W.non_hub_nodes(g))
    yield g, gh, idx
    fs.fs_graph_destroy(gh)


def _check_alone(g, gh, idx, params, steps, e, age_dtype):
    counts = fs.fs_ens_run(e, steps, len(params), 50)
    assert (g.n - counts[-1, :, 0].astype(np.int64)).min() > 50, "every realisation must have an epidemic"
    for r, p in enumerate(params):
        s = fs.fs_sim_init(gh, p, idx)
        c = fs.fs_sim_run(s, steps)
        X, A, _ = fs.fs_sim_get_state(s, g.n, age_dtype)
        fs.fs_sim_destroy(s)
        np.testing.assert_array_equal(counts[:, r, :], c, err_msg=f"realisation {r}")
        Xe, Ae, _ = fs.fs_ens_get_state(e, r, g.n, age_dtype)
        np.testing.assert_array_equal(Xe, X)
        np.testing.assert_array_equal(Ae.view(np.uint8), A.view(np.uint8))


@pytest.mark.parametrize("n_real,age_dtype,eps", [(8, fs.FS_AGE_F32, 0.0), (12, fs.FS_AGE_BF16, 0.0),
                                                  (8, fs.FS_AGE_F16, 0.03)],
                         ids=["r8-f32", "r16-bf16", "r8-f16-adaptive"])
def test_packed_shedding_equals_each_realisation_alone(hub, n_real, age_dtype, eps):
    g, gh, idx = hub
    params = realisations(n_real, age_dtype, eps)
    e = fs.fs_ens_create(gh, params, idx)
    try:
        _check_alone(g, gh, idx, params, 200, e, age_dtype)
    finally:
        fs.fs_ens_destroy(e)


def test_packed_shedding_sir_index_infectious(hub):
    """SIR with infectious index cases: the replicates' initial infectivity
    beta s(0) is written when the ensemble is created."""
    g, gh, idx = hub
    params = [shed_sir(1.5 + 0.2 * r, seed=7, replicate=r,
                       mode=fs.FS_SHED_DENSITY if r < 3 else fs.FS_SHED_HAZARD) for r in range(6)]
    e = fs.fs_ens_create(gh, params, idx)
    try:
        _check_alone(g, gh, idx, params, 120, e, fs.FS_AGE_F32)
    finally:
        fs.fs_ens_destroy(e)


def test_packed_shedding_lockstep_with_oracle(oracle_mod):
    """Each replicate of an ensemble on a Barabasi-Albert graph (merge-class
    hubs) is fed, step by step, from the ensemble's state to the oracle; the
    ensemble's next state must agree node by node except inside the band
    |u - p| < 1e-6 + dt lambda_i (d_i 2^-24 + 4e-6): FP32 sums of d_i
    non-negative terms, and infectivities evaluated in FP32 (within 4e-6
    relative of the oracle's double-precision ones, each rounded to FP32)."""
    import torch
    assert torch.cuda.is_available()
    g = W.barabasi_albert(6_000, 4, seed=13)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    assert fs.fs_graph_info_get(gh)["n_merge"] > 0
    idx = W.index_nodes(g.n, 60, seed=4, allowed=W.non_hub_nodes(g))
    params = [shed_seir(1.2, seed=19, replicate=r, mode=fs.FS_SHED_HAZARD if r < 2 else fs.FS_SHED_DENSITY)
              for r in range(4)]
    e = fs.fs_ens_create(gh, params, idx)
    deg = np.diff(g.row_ptr).astype(np.float64)
    decisions = mismatches = 0
    try:
        fs.fs_ens_run(e, 60, len(params), 50, want_counts=False)   # into the epidemic
        for _ in range(25):
            states = [fs.fs_ens_get_state(e, r, g.n) for r in range(len(params))]
            fs.fs_ens_run(e, 1, len(params), 1, want_counts=False)
            for r, p in enumerate(params):
                X, A, k = states[r]
                prm = oracle_params(oracle_mod, p)
                Xo, Ao, margin, lam = oracle_mod.step(g.row_ptr, g.col_ind, prm, k, X, A,
                                                      want_margin=True, want_lambda=True)
                X2, A2, k2 = fs.fs_ens_get_state(e, r, g.n)
                assert k2 == k + 1
                trials = np.isfinite(margin)
                decisions += int(trials.sum())
                bad = X2 != Xo
                if bad.any():
                    band = TIE + p.dt * lam[bad] * (deg[bad] * 2.0 ** -24 + 4e-6)
                    assert (np.abs(margin[bad]) < band).all(), (
                        f"replicate {r} step {k}: {int(bad.sum())} mismatches outside the band; "
                        f"margins {margin[bad][:8]}, bands {band[:8]}")
                    mismatches += int(bad.sum())
                ok = ~bad
                assert (A2[ok].view(np.uint32) == Ao[ok].view(np.uint32)).all(), f"replicate {r} step {k}: ages"
        assert decisions > 50_000
        assert mismatches <= max(2, 1e-5 * decisions), (mismatches, decisions)
    finally:
        fs.fs_ens_destroy(e)
        fs.fs_graph_destroy(gh)


def test_served_shedding_request_equals_alone(hub):
    """A request with a shedding profile served beside one without: each of
    its realisations equals the run it has alone."""
    g, gh, idx = hub
    srv = fs.fs_server_create(quantum=7)
    sc_shed = [shed_seir(1.0, seed=61, mode=fs.FS_SHED_HAZARD), shed_seir(0.8, seed=62, mode=fs.FS_SHED_DENSITY)]
    sc_plain = [fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 0.3, 0.1, 63,
                              latent=fs.law("weibull", 2.0, 4.0))]
    steps = 90
    r_plain = fs.fs_server_submit(srv, gh, sc_plain, 3, idx, steps)
    r_shed = fs.fs_server_submit(srv, gh, sc_shed, 3, idx, steps)
    fs.fs_server_drain(srv, 120)
    done, c, _ = fs.fs_server_poll(srv, r_shed, steps, 6)
    assert done
    for si, p in enumerate(sc_shed):
        for r in range(3):
            q = shed_seir(p.beta, seed=p.seed, replicate=p.replicate + r, mode=p.shed_mode)
            s = fs.fs_sim_init(gh, q, idx)
            np.testing.assert_array_equal(c[:, si * 3 + r, :], fs.fs_sim_run(s, steps))
            fs.fs_sim_destroy(s)
    done, c2, _ = fs.fs_server_poll(srv, r_plain, steps, 3)
    assert done
    s = fs.fs_sim_init(gh, fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 0.3, 0.1, 63,
                                         latent=fs.law("weibull", 2.0, 4.0), replicate=2), idx)
    np.testing.assert_array_equal(c2[:, 2, :], fs.fs_sim_run(s, steps))
    fs.fs_sim_destroy(s)
    fs.fs_server_destroy(srv)


def test_packed_shedding_argument_checks(hub):
    g, gh, idx = hub
    with pytest.raises(fs.FsError) as ex:
        fs.fs_ens_create(gh, [shed_seir(1.0, 1, mode=fs.FS_SHED_HAZARD),
                              fs.sim_params(fs.FS_SEIR, fs.law("lognormal", LN6, 0.6), 0.3, 0.1, 1,
                                            latent=fs.law("weibull", 2.0, 4.0), pressure=fs.FS_PRESSURE_GATHER)],
                         idx)
    assert ex.value.status == FS_EINVAL
    p = shed_seir(1.0, 1)
    p.flags = fs.FS_PRESSURE_PUSH
    with pytest.raises(fs.FsError) as ex:
        fs.fs_ens_create(gh, [p], idx)
    assert ex.value.status == FS_EUNSUPPORTED
