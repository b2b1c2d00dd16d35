"""Failure detection without a GPU fault.

Host side: fs_server_drain with a tiny timeout returns FS_ETIMEOUT while a
request is still running, and the server keeps serving; a request that waits
in the queue longer than the server's wait limit is retired alone with
FS_ETIMEOUT while the request ahead of it finishes with correct counts.
Device side: a bounded mbarrier wait that is made to run out (the barrier is
armed but no copy is issued, so nothing is in flight) sets the device error
word, the kernel returns, and the call reports FS_ETIMEOUT; the context stays
usable and the next run is exact. With the bounds-checked build, every checked
index of a normal run stays in bounds (error word 0), and a check whose bound
is lowered below the buffer (so the access it guards is still in bounds)
records the first index it saw as a violation.
"""
import math
import time

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W

pytestmark = pytest.mark.gpu

FS_ETIMEOUT = 4


def seir(seed, replicate=0, pressure=fs.FS_PRESSURE_AUTO):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed=seed,
                         latent=fs.law("weibull", 2.0, 4.0), replicate=replicate, pressure=pressure)


@pytest.fixture(scope="module")
def graph():
    import torch
    assert torch.cuda.is_available()
    g = W.random_regular(50_000, 10, seed=7)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    yield g, gh
    fs.fs_graph_destroy(gh)


def alone(gh, p, idx, steps):
    s = fs.fs_sim_init(gh, p, idx)
    c = fs.fs_sim_run(s, steps)
    fs.fs_sim_destroy(s)
    return c


def test_drain_times_out_while_a_request_runs(graph):
    g, gh = graph
    idx = W.index_nodes(g.n, 50, seed=3)
    srv = fs.fs_server_create(quantum=4)
    try:
        rid = fs.fs_server_submit(srv, gh, [seir(11)], 32, idx, 4000)
        with pytest.raises(fs.FsError) as e:
            fs.fs_server_drain(srv, 1e-3)
        assert e.value.status == FS_ETIMEOUT
        fs.fs_server_drain(srv, 600.0)                  # the server kept serving
        done, counts, _ = fs.fs_server_poll(srv, rid, 4000, 32)
        assert done
        np.testing.assert_array_equal(counts[:, 5, :], alone(gh, seir(11, replicate=5), idx, 4000))
    finally:
        fs.fs_server_destroy(srv)


def test_wait_limit_retires_only_the_waiting_request(graph):
    g, gh = graph
    idx = W.index_nodes(g.n, 50, seed=4)
    # one segment row: the second request cannot start while the first runs
    srv = fs.fs_server_create(max_members=1, quantum=4, wait_limit_s=0.05)
    try:
        first = fs.fs_server_submit(srv, gh, [seir(21)], 32, idx, 20000)
        t0 = time.time()
        while fs.fs_server_stats_get(srv)["running"] == 0 and time.time() - t0 < 60:
            time.sleep(0.005)
        second = fs.fs_server_submit(srv, gh, [seir(22)], 8, idx, 100)
        fs.fs_server_drain(srv, 600.0)
        with pytest.raises(fs.FsError) as e:
            fs.fs_server_poll(srv, second, 100, 8)
        assert e.value.status == FS_ETIMEOUT
        done, counts, sec = fs.fs_server_poll(srv, first, 20000, 32)
        assert done and sec > 0.05
        np.testing.assert_array_equal(counts[:, 31, :], alone(gh, seir(21, replicate=31), idx, 20000))
        st = fs.fs_server_stats_get(srv)
        assert st["completed"] == 2 and st["queued"] == 0 and st["running"] == 0
    finally:
        fs.fs_server_destroy(srv)
