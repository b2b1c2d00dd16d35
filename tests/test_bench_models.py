"""The benchmark's byte models and throughput arithmetic on hand-worked
cases (no GPU): the roofline numerators must count what the formulations
move, step by step."""
import numpy as np
import pytest

import bench


def test_push_byte_model_by_hand():
    # 12 nodes on a 4-regular graph; step 0: S 10, E 0, I 2, R 0 -> step 1:
    # S 8, E 2, I 1, R 1 (2 left S, one I recovered, no E -> I)
    counts = np.array([[10, 0, 2, 0], [8, 2, 1, 1]], dtype=np.uint32)
    got = bench.push_bytes_model(counts, 12, 4)
    # states 12 x 1 + S counts/tallies 10 x 3 + E/I ages 2 x 2 x 4 + 3 state
    # writes + one pushing node (row bounds 16 + 4 out-edges x 8)
    assert got.shape == (1,)
    assert got[0] == 12 + 30 + 16 + 3 + (16 + 32)


def test_push_byte_model_counts_entries_to_i():
    # SEIR: E -> I for 3 nodes and I -> R for 1 in the same step
    counts = np.array([[50, 5, 4, 1], [48, 4, 6, 2]], dtype=np.uint32)
    got = bench.push_bytes_model(counts, 60, 10, b_age=2)
    left_s, to_r = 2, 1
    enter_i = (6 - 4) + to_r            # I grew by 2 while 1 left it: 3 entered
    pushers = enter_i + to_r
    want = 60 + 3 * 50 + 2 * 2 * (5 + 4) + (left_s + enter_i + to_r) + pushers * (16 + 10 * 8)
    assert got[0] == want


def test_pull_byte_model_by_hand():
    # 100 nodes, 3 steps, 150 S node-steps with 1,200 S-row edges
    got = bench.bytes_model(100, 3, 150, 1200)
    assert got == pytest.approx(100 * 3 * (2 + 8 + 0.125) + 4 * 150 + 4.125 * 1200)
    got16 = bench.bytes_model(100, 3, 150, 1200, b_age=2)
    assert got - got16 == pytest.approx(100 * 3 * 4)


def test_whole_job_throughput():
    # 10^6 nodes x 1,000 steps x 5 benchmark steps x 2 replicas in 100 ms
    assert bench.whole_job_gnups(1_000_000, 1000, 5, 2, 100.0) == pytest.approx(100.0)


def test_host_oracle_pool_steps_independent_realisations():
    """The CPU baseline's pool: every worker is the oracle on its own
    replicate, and its realisation equals the oracle run directly."""
    import math
    import oracle as om
    import workloads as W
    g = W.random_regular(3000, 6, seed=2)
    idx = W.index_nodes(g.n, 30, seed=3)
    h = bench.HostOracle(g, idx, workers=2)
    try:
        upd, wall, steps = h.advance(12)
        assert steps == [12, 12] and upd == g.n * 24 and wall > 0
        got = h.counts()
    finally:
        h.close()
    for rep, (k, c) in enumerate(got):
        prm = om.params(om.SEIR, om.law("weibull", 2.0, 4.0), om.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1,
                        seed=1, rep=rep)
        X, A = om.init(g.n, idx, om.E)
        ref, _, _ = om.run(g.row_ptr, g.col_ind, prm, 0, 12, X, A)
        assert k == 12
        assert c == ref[-1].tolist()
    assert got[0][1] != got[1][1], "the two replicates must draw different uniforms"


def test_breq_of_a_push_trajectory():
    # 3 steps on a 10-regular graph of 100 nodes: S at the start of each step
    # 90, 80, 75 (row 3 is the state after the last step)
    counts = np.array([[90, 5, 5, 0], [80, 10, 8, 2], [75, 10, 10, 5], [70, 9, 11, 10]], dtype=np.uint32)
    got = bench.breq_regular(counts, 100, 10)
    s = 90 + 80 + 75
    assert got == pytest.approx(3 * 100 * (2 + 8 + 0.125) + 4 * s + 4.125 * 10 * s)
