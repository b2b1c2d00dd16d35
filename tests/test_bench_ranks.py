"""The multi-rank path of bench.py (replicas only: one replica per GPU, no
data-path collective) on CPU: rank/world setup from torchrun's environment,
the max over ranks of the timed region through a world_size-2 gloo group,
the whole-job value, and distinct replica seeds."""
import multiprocessing as mp
import os
import socket

import pytest

import bench


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, local_ms: list, q):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, w, lr, changes = bench.rank_setup(os.environ, 1)
    dist.init_process_group("gloo", rank=r, world_size=w)
    m = bench.max_over_ranks(local_ms[r], dist, torch.device("cpu"))
    v = bench.whole_job_gnups(1000, 10, 2, w, m)
    dist.barrier()
    q.put((r, w, lr, changes, m, v, bench.replica_seed(r)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    local_ms = [3.0, 5.0]
    ps = [ctx.Process(target=_rank, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, lr, changes, m, v, seed) in enumerate(out):
        assert (rank, w, lr) == (r, 2, 0)
        assert changes == {"CUDA_VISIBLE_DEVICES": str(r), "LOCAL_RANK": "0"}
        assert m == 5.0                                     # the slowest rank's time on every rank
        assert v == pytest.approx(1000 * 10 * 2 * 2 / 5e-3 / 1e9)
    assert out[0][6] != out[1][6]                           # distinct replicas


def test_single_process_defaults():
    assert bench.rank_setup({}, 1) == (0, 1, 0, {})
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_gnups(10**6, 1000, 5, 1, 10.0 * 5) == pytest.approx(100.0)
