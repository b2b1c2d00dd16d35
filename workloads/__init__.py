"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input generation only: contact graphs (random d-regular by
the configuration model with repair, Erdos-Renyi G(n, p), Barabasi-Albert),
index-case lists and scenario draws. It contains none of the epidemic
method's arithmetic and imports neither the CUDA library nor the oracle, so
both sides of every parity test read identical inputs from here.

All randomness comes from splitmix64 streams (Steele, Lea, Flood 2014) keyed
by an explicit seed, so the same seed gives the same graph on any machine and
any numpy version. Graphs are returned as undirected CSR, row i listing the
neighbours of i sorted ascending: row_ptr int64[n+1], col_ind int32[2m].
The paper's workloads are synthetic graphs of these families (FlashSpread,
arXiv 2604.22092, Section 6 and Appendix C.4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """`count` consecutive outputs of splitmix64 started at state seed ^ stream."""
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) ^ (int(stream) * 0xD1B54A32D192ED03)) & 0xFFFFFFFFFFFFFFFF)
        z = base + _GOLDEN * (np.arange(1, count + 1, dtype=np.uint64))
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_below(seed: int, bounds: np.ndarray, stream: int) -> np.ndarray:
    """Integers uniform in [0, bounds[i]) (multiply-shift on 64-bit draws)."""
    bounds = np.asarray(bounds, dtype=np.uint64)
    r = splitmix64(seed, bounds.size, stream)
    hi = (r >> np.uint64(32))
    lo = (r & np.uint64(0xFFFFFFFF))
    # floor(r * b / 2^64) computed in two 32-bit halves
    b_hi = bounds >> np.uint64(32)
    b_lo = bounds & np.uint64(0xFFFFFFFF)
    with np.errstate(over="ignore"):
        t = lo * b_lo
        mid = hi * b_lo + (t >> np.uint64(32))
        mid2 = lo * b_hi + (mid & np.uint64(0xFFFFFFFF))
        res = hi * b_hi + (mid >> np.uint64(32)) + (mid2 >> np.uint64(32))
    return res.astype(np.int64)


def uniform01(seed: int, count: int, stream: int) -> np.ndarray:
    return (splitmix64(seed, count, stream) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def permutation(seed: int, n: int, stream: int) -> np.ndarray:
    """A random permutation of range(n): argsort of splitmix64 keys."""
    return np.argsort(splitmix64(seed, n, stream), kind="stable").astype(np.int64)


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray   # int64 [n+1]
    col_ind: np.ndarray   # int32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, name: str = "") -> Graph:
    """Undirected simple edge list (u, v), u != v, no repeats -> symmetric CSR."""
    src = np.concatenate([u, v]).astype(np.int64)
    dst = np.concatenate([v, u]).astype(np.int64)
    key = src * np.int64(n) + dst
    key.sort(kind="stable")
    rows = key // np.int64(n)
    cols = (key - rows * np.int64(n)).astype(np.int32)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n, row_ptr, cols, name)


def empty_graph(n: int) -> Graph:
    return Graph(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), "empty")


def _bad_pairs(n: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Mask of pairs that are self-loops or repeats of an earlier pair."""
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = lo * np.int64(n) + hi
    order = np.argsort(key, kind="stable")
    ks = key[order]
    dup_sorted = np.zeros(ks.size, dtype=bool)
    dup_sorted[1:] = ks[1:] == ks[:-1]
    dup = np.zeros(ks.size, dtype=bool)
    dup[order] = dup_sorted
    return dup | (a == b)


def random_regular(n: int, d: int, seed: int) -> Graph:
    """Random simple d-regular graph: configuration model (uniform stub pairing)
    followed by repair of self-loops and repeated edges by re-pairing the
    offending stubs together with randomly chosen good pairs until none is left."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    stubs = stubs[permutation(seed, stubs.size, stream=1)]
    a = stubs[0::2].copy()
    b = stubs[1::2].copy()
    m = a.size
    rnd = 2
    while True:
        bad = np.flatnonzero(_bad_pairs(n, a, b))
        if bad.size == 0:
            break
        if rnd > 200:
            raise RuntimeError("random_regular: repair did not converge")
        # re-pair the stubs of the bad edges with those of as many random edges
        extra = uniform_below(seed, np.full(max(bad.size, 4), m, dtype=np.uint64), stream=1000 + rnd)
        sel = np.unique(np.concatenate([bad, extra]))
        pool = np.concatenate([a[sel], b[sel]])
        pool = pool[permutation(seed, pool.size, stream=5000 + rnd)]
        a[sel] = pool[0::2]
        b[sel] = pool[1::2]
        rnd += 1
    return csr_from_edges(n, a, b, name=f"regular(n={n},d={d},seed={seed})")


def erdos_renyi(n: int, mean_degree: float, seed: int) -> Graph:
    """G(n, p), p = mean_degree/(n-1), by geometric skipping over the n(n-1)/2
    unordered pairs (Batagelj and Brandes 2005)."""
    p = mean_degree / (n - 1)
    total = n * (n - 1) // 2
    expect = int(total * p)
    chunk = max(1024, int(expect + 8 * math.sqrt(expect + 1) + 64))
    gaps_all = []
    pos = -1
    stream = 3
    while True:
        u = uniform01(seed, chunk, stream)
        u = np.clip(u, 1e-300, 1.0)
        gaps = np.floor(np.log(u) / math.log1p(-p)).astype(np.int64) + 1
        cs = pos + np.cumsum(gaps)
        keep = cs < total
        gaps_all.append(cs[keep])
        if not keep.all():
            break
        pos = int(cs[-1])
        stream += 1
    L = np.concatenate(gaps_all)
    # unrank L -> (i, j), i < j, row-major over the strict upper triangle
    # row i starts at s(i) = i*(2n-i-1)/2
    i = np.floor((2 * n - 1 - np.sqrt((2.0 * n - 1) ** 2 - 8.0 * L)) / 2).astype(np.int64)
    i = np.clip(i, 0, n - 2)
    s = i * (2 * n - i - 1) // 2
    over = s > L
    while over.any():
        i[over] -= 1
        s = i * (2 * n - i - 1) // 2
        over = s > L
    nxt = (i + 1) * (2 * n - i - 2) // 2
    under = nxt <= L
    while under.any():
        i[under] += 1
        s = i * (2 * n - i - 1) // 2
        nxt = (i + 1) * (2 * n - i - 2) // 2
        under = nxt <= L
    j = L - s + i + 1
    return csr_from_edges(n, i, j, name=f"er(n={n},d={mean_degree},seed={seed})")


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    """Preferential attachment: a clique on m+1 nodes, then every new node v
    attaches to m distinct earlier nodes chosen with probability proportional
    to degree, drawn as uniform positions in the endpoint list of the edges
    that exist before v (the repeated-node list of Batagelj and Brandes).

    All positions are drawn at once and resolved by pointer doubling (a
    position that holds an earlier node's target points at that target's
    slot); a node whose m targets repeat redraws the later copies and the
    whole list is resolved again, which equals the sequential process."""
    if n <= m + 1:
        raise ValueError("n must exceed m+1")
    c = m + 1
    cu, cv = np.triu_indices(c, k=1)
    E0 = cu.size
    nv = n - c
    clique_ep = np.empty(2 * E0, dtype=np.int64)
    clique_ep[0::2] = cu
    clique_ep[1::2] = cv
    slots = nv * m
    vi = np.arange(slots, dtype=np.int64) // m
    base_len = (2 * (E0 + vi * m)).astype(np.uint64)   # endpoints before node c+vi
    pos = uniform_below(seed, base_len, stream=7000)
    rnd = 1
    while True:
        val = np.full(slots, -1, dtype=np.int64)
        ptr = np.full(slots, -1, dtype=np.int64)
        inc = pos < 2 * E0
        val[inc] = clique_ep[pos[inc]]
        q = pos[~inc] - 2 * E0
        slot = q // 2
        even = (q % 2) == 0
        idx = np.flatnonzero(~inc)
        val[idx[even]] = c + slot[even] // m
        ptr[idx[~even]] = slot[~even]
        un = np.flatnonzero(val < 0)
        while un.size:
            p = ptr[un]
            got = val[p] >= 0
            val[un[got]] = val[p[got]]
            ptr[un[~got]] = ptr[p[~got]]
            un = un[~got]
        targets = val.reshape(nv, m)
        order = np.argsort(targets, axis=1, kind="stable")
        srt = np.take_along_axis(targets, order, axis=1)
        dupl_sorted = np.zeros_like(srt, dtype=bool)
        dupl_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
        if not dupl_sorted.any():
            break
        # the later slot of each repeated pair is redrawn
        r_, k_ = np.nonzero(dupl_sorted)
        a_slot = order[r_, k_]
        b_slot = order[r_, k_ - 1]
        redo = r_ * m + np.maximum(a_slot, b_slot)
        redo = np.unique(redo)
        pos[redo] = uniform_below(seed, base_len[redo], stream=7000 + rnd)
        rnd += 1
        if rnd > 10_000:
            raise RuntimeError("barabasi_albert: did not converge")
    v = np.arange(c, n, dtype=np.int64)
    u = np.concatenate([cu.astype(np.int64), np.repeat(v, m)])
    w = np.concatenate([cv.astype(np.int64), targets.reshape(-1)])
    return csr_from_edges(n, u, w, name=f"ba(n={n},m={m},seed={seed})")


def index_nodes(n: int, count: int, seed: int, allowed: np.ndarray | None = None) -> np.ndarray:
    """`count` distinct node ids drawn uniformly without replacement from
    `allowed` (default: all nodes), by Floyd's algorithm on splitmix64 draws."""
    pool = np.arange(n, dtype=np.int64) if allowed is None else np.asarray(allowed, dtype=np.int64)
    M = pool.size
    if count > M:
        raise ValueError("more index nodes than candidates")
    draws = uniform_below(seed ^ 0x1D, np.arange(M - count + 1, M + 1, dtype=np.uint64), stream=11)
    chosen: list[int] = []
    seen: set[int] = set()
    for t, j in zip(range(M - count, M), draws):
        r = int(j)
        pick = r if r not in seen else t
        seen.add(pick)
        chosen.append(pick)
    return np.sort(pool[np.array(chosen, dtype=np.int64)]).astype(np.int32)


def non_hub_nodes(g: Graph) -> np.ndarray:
    """Nodes of degree at most ceil(mean degree)."""
    deg = g.degree
    return np.flatnonzero(deg <= math.ceil(deg.mean())).astype(np.int64)


# ---------------------------------------------------------------- ensembles
@dataclass
class Scenario:
    """Parameters of one realisation drawn for the ensemble and serving
    workloads: beta ~ U[0.1, 0.5]; infectious log-normal with mu = ln 6 and
    sigma ~ U[0.3, 1.0]; latent Erlang(3, rate 0.75/d, mean 4 d) for even
    scenario indices and Weibull(2, 4 d) for odd ones."""
    beta: float
    sigma_inf: float
    latent: str            # "erlang" or "weibull"
    seed: int


def scenarios(count: int, seed: int) -> list[Scenario]:
    u = uniform01(seed, 2 * count, stream=91)
    return [Scenario(0.1 + 0.4 * u[2 * s], 0.3 + 0.7 * u[2 * s + 1], "erlang" if s % 2 == 0 else "weibull",
                     int(seed * 1_000_003 + s) & 0xFFFFFFFFFFFF) for s in range(count)]


def mixed_graph(q: int, n_lo: float, n_hi: float, seed: int) -> Graph:
    """Graph q of a mixed ensemble: N log-uniform in [n_lo, n_hi]; the family
    cycles random-regular (k uniform in 4..20), Erdos-Renyi (mean degree 8)
    and Barabasi-Albert (m uniform in 2..8); graph seed q."""
    u = uniform01(seed, 3, stream=300 + q)
    n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
    fam = q % 3
    if fam == 0:
        k = 4 + int(u[1] * 17)
        if (n * k) % 2:
            n += 1
        return random_regular(n, k, seed=q)
    if fam == 1:
        return erdos_renyi(n, 8.0, seed=q)
    m = 2 + int(u[2] * 7)
    return barabasi_albert(n, m, seed=q)


@dataclass
class Request:
    arrival: float         # seconds after the start
    graph: int             # index into the graph pool
    n_scen: int
    replicates: int
    steps: int
    seed: int


def request_stream(count: int, rate_per_s: float, n_graphs: int, seed: int, steps: int = 200,
                   rep_lo: int = 16, rep_hi: int = 256) -> list[Request]:
    """Poisson arrivals (exponential gaps at `rate_per_s`); each request picks
    a pooled graph uniformly, 1..4 scenarios and a replicate count
    log-uniform in [rep_lo, rep_hi]."""
    u = uniform01(seed, 4 * count, stream=404)
    t = 0.0
    out = []
    for r in range(count):
        t += -math.log(max(u[4 * r], 1e-12)) / rate_per_s
        reps = int(round(math.exp(math.log(rep_lo) + u[4 * r + 1] * (math.log(rep_hi) - math.log(rep_lo)))))
        out.append(Request(t, int(u[4 * r + 2] * n_graphs), 1 + int(u[4 * r + 3] * 4), reps, steps,
                           seed * 7919 + r))
    return out
