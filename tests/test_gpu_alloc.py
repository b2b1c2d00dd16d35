"""Device memory: the library's caching allocator and a caller's allocator.

With fs_set_allocator every block of a graph, a simulation, an ensemble and
a batch comes from the caller's functions (here PyTorch's caching allocator)
and goes back through them, and results are identical to those with the
library's own allocator. The library's allocator keeps freed blocks (cached
bytes grow when objects are destroyed, and the next object of the same size
reuses them) until fs_release_cached_memory.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W

pytestmark = pytest.mark.gpu


def seir(seed, replicate=0, pressure=fs.FS_PRESSURE_AUTO):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed=seed,
                         latent=fs.law("weibull", 2.0, 4.0), replicate=replicate, pressure=pressure)


def run_all(g, idx):
    """A push-form and a gather-form sim and a packed ensemble in a batch:
    their counts."""
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    out = []
    for pr in (fs.FS_PRESSURE_PUSH, fs.FS_PRESSURE_GATHER):
        s = fs.fs_sim_init(gh, seir(5, pressure=pr), idx)
        out.append(fs.fs_sim_run(s, 200))
        fs.fs_sim_destroy(s)
    e = fs.fs_ens_create(gh, [seir(7, replicate=r) for r in range(8)], idx)
    b = fs.fs_batch_create(fs.FS_AGE_F32, 4)
    counts = np.zeros((201, 8, 4), dtype=np.uint32)
    fs.fs_batch_add(b, e, 200, counts)
    fs.fs_batch_run(b, 201, 50)
    out.append(counts.copy())
    fs.fs_batch_destroy(b)
    fs.fs_ens_destroy(e)
    fs.fs_graph_destroy(gh)
    return out


def test_caller_allocator_serves_every_block():
    import torch
    assert torch.cuda.is_available()
    g = W.barabasi_albert(30_000, 4, seed=11)
    idx = W.index_nodes(g.n, 20, seed=2, allowed=W.non_hub_nodes(g))
    ref = run_all(g, idx)
    live, calls = {}, {"alloc": 0, "free": 0, "peak": 0}

    def alloc(nbytes):
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        calls["alloc"] += 1
        calls["peak"] = max(calls["peak"], len(live))
        return t.data_ptr()

    def free(ptr):
        del live[ptr]
        calls["free"] += 1

    fs.fs_set_allocator(alloc, free)
    try:
        got = run_all(g, idx)
    finally:
        fs.fs_set_allocator(None, None)
    assert calls["alloc"] > 10 and calls["alloc"] == calls["free"] and not live, calls
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(ValueError):
        fs.fs_set_allocator(alloc, None)


def test_library_allocator_caches_and_releases():
    import torch
    assert torch.cuda.is_available()
    g = W.random_regular(200_000, 10, seed=4)
    idx = W.index_nodes(g.n, 20, seed=1)
    fs.fs_release_cached_memory()
    assert fs.fs_cached_memory()["cached_bytes"] == 0
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, seir(3), idx)
    c1 = fs.fs_sim_run(s, 100)
    live = fs.fs_cached_memory()["live_blocks"]
    assert live > 0
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
    cached = fs.fs_cached_memory()["cached_bytes"]
    assert cached > g.nnz * 4                       # at least the columns' blocks were kept
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    s = fs.fs_sim_init(gh, seir(3), idx)
    assert fs.fs_cached_memory()["cached_bytes"] < cached   # the same sizes were handed out again
    np.testing.assert_array_equal(fs.fs_sim_run(s, 100), c1)
    fs.fs_sim_destroy(s)
    fs.fs_graph_destroy(gh)
    fs.fs_release_cached_memory()
    assert fs.fs_cached_memory()["cached_bytes"] == 0
