"""The dispatch autotuner (FS_DISPATCH_TUNE): it times every candidate class
split of a skewed graph, keeps one of them, caches the choice per degree
profile, needs no trial for graphs that fit one class, and never changes
results (every split is bit-identical)."""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W

pytestmark = pytest.mark.gpu


def seir(seed=5):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0))


def counts(gh, idx, steps):
    s = fs.fs_sim_init(gh, seir(), idx)
    c = fs.fs_sim_run(s, steps)
    fs.fs_sim_destroy(s)
    return c


def test_tune_picks_a_candidate_caches_it_and_keeps_results():
    import torch
    assert torch.cuda.is_available()
    fs.load()
    fs.fs_tune_reset()
    g = W.barabasi_albert(200_000, 5, seed=21)
    idx = W.index_nodes(g.n, 50, seed=22, allowed=W.non_hub_nodes(g))
    auto = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    tuned = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(dispatch=fs.FS_DISPATCH_TUNE))
    ia, it = fs.fs_graph_info_get(auto), fs.fs_graph_info_get(tuned)
    assert ia["d_max"] > 255
    assert it["thread_max_deg"] in (31, 63, 127, 255)
    st = fs.fs_tune_stats()
    assert st == {"trials": 4, "cache_hits": 0, "profiles": 1}
    np.testing.assert_array_equal(counts(tuned, idx, 150), counts(auto, idx, 150))
    # same degree profile: answered from the cache, same split
    g2 = W.barabasi_albert(200_000, 5, seed=23)
    t2 = fs.fs_graph_create(g2.n, g2.row_ptr, g2.col_ind, opts=fs.graph_opts(dispatch=fs.FS_DISPATCH_TUNE))
    i2 = fs.fs_graph_info_get(t2)
    if i2["d_max"] > 255 and math.ceil(math.log2(i2["d_max"])) == math.ceil(math.log2(ia["d_max"])):
        assert fs.fs_tune_stats()["cache_hits"] == 1
        assert fs.fs_tune_stats()["trials"] == 4
        assert i2["thread_max_deg"] == it["thread_max_deg"]
    # a graph that fits one class needs no trial
    r = W.random_regular(50_000, 10, seed=24)
    tr = fs.fs_graph_create(r.n, r.row_ptr, r.col_ind, opts=fs.graph_opts(dispatch=fs.FS_DISPATCH_TUNE))
    assert fs.fs_graph_info_get(tr)["n_merge"] == 0
    assert fs.fs_tune_stats()["trials"] == 4
    with pytest.raises(fs.FsError):
        fs.fs_graph_create(g.n, g.row_ptr, g.col_ind,
                           opts=fs.graph_opts(dispatch=fs.FS_DISPATCH_TUNE, thread_max_deg=63))
    for h in (auto, tuned, t2, tr):
        fs.fs_graph_destroy(h)
    fs.fs_tune_reset()
    assert fs.fs_tune_stats() == {"trials": 0, "cache_hits": 0, "profiles": 0}
