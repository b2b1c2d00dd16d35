"""Age storage precision, stated per result (FP16 / BF16 against FP32, whose
trajectories are the FP64 oracle's). Replicates keep their random streams
under every storage type, so the paired differences of their peak infectious
fraction and attack rate isolate the storage. Reduced-precision ensembles are
also compared with the oracle run at the same storage (it emulates the
rounding exactly), replicate by replicate."""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W
from tests.gpu_helpers import oracle_params

pytestmark = pytest.mark.gpu

STORAGE = {"f32": fs.FS_AGE_F32, "f16": fs.FS_AGE_F16, "bf16": fs.FS_AGE_BF16}


def ensemble_counts(gh, idx, beta, steps, reps, age):
    lat, inf = fs.law("weibull", 2.0, 4.0), fs.law("lognormal", math.log(6.0), 0.6)
    prm = [fs.sim_params(fs.FS_SEIR, inf, beta, 0.1, 3, latent=lat, replicate=r, age_dtype=age) for r in range(reps)]
    b = fs.fs_batch_create(age, reps // 32 + 2)
    ens, outs = [], []
    for off in range(0, reps, 32):
        e = fs.fs_ens_create(gh, prm[off:off + 32], idx)
        o = np.zeros((steps + 1, min(32, reps - off), 4), dtype=np.uint32)
        fs.fs_batch_add(b, e, steps, o)
        ens.append(e)
        outs.append(o)
    fs.fs_batch_run(b, steps + 1, 50)
    fs.fs_batch_destroy(b)
    for e in ens:
        fs.fs_ens_destroy(e)
    return np.concatenate(outs, axis=1).astype(np.int64), prm


@pytest.mark.parametrize("beta", [0.25, 0.05])
def test_storage_shifts_are_small_and_exact_against_the_oracle(beta, oracle_mod):
    import torch
    assert torch.cuda.is_available()
    fs.load()
    g = W.random_regular(20_000, 10, seed=12)
    idx = W.index_nodes(g.n, 30, seed=13)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    steps, reps = 800, 96
    peak, attack = {}, {}
    for name, age in STORAGE.items():
        c, prm = ensemble_counts(gh, idx, beta, steps, reps, age)
        assert (c.sum(axis=2) == g.n).all()
        peak[name] = c[:, :, 2].max(axis=0) / g.n
        attack[name] = 1.0 - c[-1, :, 0] / g.n
        for r in (0, 57):                       # this storage's trajectory == the oracle at this storage
            X0, A0 = oracle_mod.init(g.n, idx, oracle_mod.E)
            ref, _, _ = oracle_mod.run(g.row_ptr, g.col_ind, oracle_params(oracle_mod, prm[r]), 0, steps, X0, A0)
            np.testing.assert_array_equal(c[:, r, :], ref, err_msg=f"{name} replicate {r}")
    fs.fs_graph_destroy(gh)
    assert attack["f32"].mean() > (0.9 if beta == 0.25 else 0.05)
    for name in ("f16", "bf16"):
        dp = peak[name] - peak["f32"]
        da = attack[name] - attack["f32"]
        # storage moves each result by well under a percentage point
        assert abs(dp.mean()) < 5e-3, (name, dp.mean())
        assert abs(da.mean()) < 1e-2, (name, da.mean())
