"""The seeded synthetic inputs (workloads/) have the structure their recipe
states: random d-regular graphs are simple and exactly d-regular; Erdos-Renyi
graphs are simple with the binomial edge count of G(n, p); Barabasi-Albert
graphs grow from an (m+1)-clique with m distinct earlier targets per node and
a heavy degree tail; CSR rows are symmetric; index cases are distinct, in
range and drawn from the allowed pool, uniformly; the scenario and request
generators stay inside their stated ranges; everything is reproducible from
its seed."""
import math

import numpy as np
import pytest

import workloads as W


def edges(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return rows, g.col_ind.astype(np.int64)


def assert_simple_symmetric(g):
    u, v = edges(g)
    assert (u != v).all(), "self-loop"
    key = u * g.n + v
    assert np.unique(key).size == key.size, "repeated edge"
    rev = np.sort(v * g.n + u)
    np.testing.assert_array_equal(np.sort(key), rev)     # every edge listed both ways


@pytest.mark.parametrize("n,d", [(1000, 4), (2001, 10), (5000, 8)])
def test_random_regular_is_simple_and_regular(n, d):
    if (n * d) % 2:
        n += 1
    g = W.random_regular(n, d, seed=3)
    assert g.n == n
    assert (np.diff(g.row_ptr) == d).all()
    assert_simple_symmetric(g)


def test_erdos_renyi_edge_count_and_simplicity():
    n, md = 20_000, 8.0
    g = W.erdos_renyi(n, md, seed=5)
    assert_simple_symmetric(g)
    m = g.col_ind.size // 2
    pairs = n * (n - 1) // 2
    p = md / (n - 1)
    z = (m - pairs * p) / math.sqrt(pairs * p * (1 - p))
    assert abs(z) < 5, z
    # degrees are binomial(n - 1, p): mean and variance
    deg = np.diff(g.row_ptr)
    assert abs(deg.mean() - md) < 0.1
    assert abs(deg.var() / (md * (1 - p)) - 1) < 0.05


def test_barabasi_albert_structure():
    n, m = 30_000, 4
    g = W.barabasi_albert(n, m, seed=9)
    assert_simple_symmetric(g)
    deg = np.diff(g.row_ptr)
    assert g.col_ind.size // 2 == m * (m + 1) // 2 + (n - m - 1) * m
    assert deg.min() >= m
    # the seed clique: nodes 0..m are all joined
    for a in range(m + 1):
        row = set(g.col_ind[g.row_ptr[a]:g.row_ptr[a + 1]].tolist())
        assert set(range(m + 1)) - {a} <= row
    # every later node joined m distinct earlier nodes
    u, v = edges(g)
    later = u >= m + 1
    earlier_targets = np.bincount(u[later & (v < u)], minlength=n)[m + 1:]
    assert (earlier_targets == m).all()
    # preferential attachment: a heavy tail (max degree far above the mean)
    assert deg.max() > 20 * deg.mean()


def test_index_nodes_distinct_in_pool_and_uniform():
    n = 1000
    counts = np.zeros(n)
    allowed = np.arange(0, n, 2)
    for s in range(400):
        idx = W.index_nodes(n, 25, seed=s, allowed=allowed)
        assert idx.size == 25 and np.unique(idx).size == 25
        assert (idx % 2 == 0).all() and (idx < n).all()
        counts[idx] += 1
    # each allowed node is picked 400 * 25 / 500 = 20 times on average
    c = counts[allowed]
    chi2 = ((c - 20.0) ** 2 / 20.0).sum()
    assert chi2 < 500 + 5 * math.sqrt(2 * 499), chi2
    assert counts[1::2].sum() == 0


def test_scenarios_and_requests_in_range():
    sc = W.scenarios(64, seed=1000)
    assert all(0.1 <= s.beta <= 0.5 and 0.3 <= s.sigma_inf <= 1.0 for s in sc)
    assert [s.latent for s in sc[:4]] == ["erlang", "weibull", "erlang", "weibull"]
    reqs = W.request_stream(500, 40.0, 16, seed=3)
    t = np.array([r.arrival for r in reqs])
    assert (np.diff(t) > 0).all()
    # Poisson arrivals at 40/s: mean gap 1/40 s
    assert abs(np.diff(t).mean() * 40 - 1) < 0.15
    assert all(16 <= r.replicates <= 256 and 1 <= r.n_scen <= 4 and 0 <= r.graph < 16 for r in reqs)


def test_mixed_family_sizes_and_kinds():
    for q in range(6):
        g = W.mixed_graph(q, 1e4, 3e4, seed=2026)
        assert 1e4 <= g.n <= 3e4 + 1
        assert_simple_symmetric(g)
    # the family cycles regular (q % 3 == 0: one degree), Erdos-Renyi, Barabasi-Albert
    assert np.diff(W.mixed_graph(3, 1e4, 3e4, seed=2026).row_ptr).std() == 0
    ba = np.diff(W.mixed_graph(5, 1e4, 3e4, seed=2026).row_ptr)
    assert ba.max() > 10 * ba.mean()


def test_generators_are_reproducible():
    a, b = W.barabasi_albert(5000, 3, seed=4), W.barabasi_albert(5000, 3, seed=4)
    np.testing.assert_array_equal(a.col_ind, b.col_ind)
    c = W.barabasi_albert(5000, 3, seed=5)
    assert not np.array_equal(a.col_ind, c.col_ind)
    np.testing.assert_array_equal(W.index_nodes(10_000, 100, seed=1), W.index_nodes(10_000, 100, seed=1))
