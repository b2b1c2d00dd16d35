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
from tests.gpu_helpers import lockstep

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


FS_ESTATE = 6
FS_ECUDA = 3


def test_bounded_device_wait_runs_out_and_reports_timeout(oracle_mod):
    """The gather form's merge chunks wait (bounded) on an mbarrier for their
    bulk copy. With the test setting the barrier is armed but no copy is
    issued, so every wait runs out with nothing in flight: the step records
    the error word and returns, the run reports FS_ETIMEOUT, the sim refuses
    further work (FS_ESTATE), and the graph and the context stay usable."""
    g = W.barabasi_albert(30_000, 4, seed=9)
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    try:
        assert fs.fs_graph_info_get(gh)["n_merge"] > 0
        idx = W.index_nodes(g.n, 30, seed=5, allowed=W.non_hub_nodes(g))
        p = seir(31, pressure=fs.FS_PRESSURE_GATHER)
        fs.fs_test_inject(fs.FS_TEST_WAIT_TIMEOUT, 64)
        try:
            s = fs.fs_sim_init(gh, p, idx)
        finally:
            fs.fs_test_inject(fs.FS_TEST_WAIT_TIMEOUT, 0)
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_run(s, 5, graph_steps=5)
        assert e.value.status == FS_ETIMEOUT and "bounded device wait" in str(e.value)
        with pytest.raises(fs.FsError) as e:
            fs.fs_sim_run(s, 1)
        assert e.value.status == FS_ESTATE
        fs.fs_sim_destroy(s)
        s = fs.fs_sim_init(gh, p, idx)        # created after the setting was turned off
        lockstep(oracle_mod, g, p, s, 5)
        fs.fs_sim_destroy(s)
    finally:
        fs.fs_graph_destroy(gh)


BOUNDS_CHILD = r"""
import math, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2604_22092_gb300 as fs
import oracle as om
import workloads as W
assert fs.fs_debug_bounds_build(), "the bounds-checked library must be loaded"
om.build()
g = W.random_regular(10_000, 10, seed=0)
idx = W.index_nodes(g.n, 10, seed=1)
gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
prm = om.params(om.SIR, None, om.law("lognormal", math.log(5.0), 0.5), 0.3, 0.1, seed=1)
X0, A0 = om.init(g.n, idx, om.I)
ref, _, _ = om.run(g.row_ptr, g.col_ind, prm, 0, 300, X0, A0)
for pressure in (fs.FS_PRESSURE_PUSH, fs.FS_PRESSURE_GATHER):
    p = fs.sim_params(fs.FS_SIR, fs.law("lognormal", math.log(5.0), 0.5), 0.3, 0.1, seed=1, pressure=pressure)
    s = fs.fs_sim_init(gh, p, idx)
    c = fs.fs_sim_run(s, 300, graph_steps=50)      # every checked index in range: no error word
    assert np.array_equal(c, ref), pressure
    fs.fs_sim_destroy(s)
ba = W.barabasi_albert(20_000, 4, seed=3)
hb = fs.fs_graph_create(ba.n, ba.row_ptr, ba.col_ind)
for pressure in (fs.FS_PRESSURE_PUSH, fs.FS_PRESSURE_GATHER):
    p = fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed=2,
                      latent=fs.law("weibull", 2.0, 4.0), pressure=pressure)
    s = fs.fs_sim_init(hb, p, W.index_nodes(ba.n, 20, seed=4, allowed=W.non_hub_nodes(ba)))
    fs.fs_sim_run(s, 400, graph_steps=50)
    fs.fs_sim_destroy(s)
fs.fs_graph_destroy(hb)
# the transposed CSR's column check put 7 entries before the buffer's end:
# the first push to read one of the last 7 columns is rejected and reported
nnz = int(g.row_ptr[-1])
fs.fs_test_inject(fs.FS_TEST_BOUNDS_SHRINK, 7)
try:
    p = fs.sim_params(fs.FS_SIR, fs.law("lognormal", math.log(5.0), 0.5), 0.3, 0.1, seed=1,
                      pressure=fs.FS_PRESSURE_PUSH)
    s = fs.fs_sim_init(gh, p, idx)
finally:
    fs.fs_test_inject(fs.FS_TEST_BOUNDS_SHRINK, 0)
try:
    fs.fs_sim_run(s, 300, graph_steps=50)
    raise SystemExit("the lowered bound was not reported")
except fs.FsError as e:
    msg = str(e)
    assert e.status == 3 and "bounds check failed: site 3," in msg, msg
    index = int(msg.split("index ")[1].split(" ")[0])
    assert nnz - 7 <= index < nnz, (index, nnz)
fs.fs_sim_destroy(s)
fs.fs_graph_destroy(gh)
print("BOUNDS_OK")
"""


def test_bounds_checked_build():
    """The FS_DEBUG_BOUNDS build (a separate library, loaded in a child
    process): normal runs of both pressure forms, with SELL slices, merge
    chunks and pushes, trip no check and equal the oracle; a check whose bound
    is lowered below the buffer's end reports the first index it rejects."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FLASHSTEP_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", BOUNDS_CHILD, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "BOUNDS_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
