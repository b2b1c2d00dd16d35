#!/usr/bin/env python3
"""Benchmark of the fused renewal tau-leaping step (GNUPS = N * steps / time).

One benchmark step is one whole run of the SEIR workload on a random
10-regular graph with N = 10^6 (Weibull(2, 4 d) latent period, log-normal
(ln 6, 0.6) infectious period, beta = 0.25/day, 100 uniformly chosen index
cases, dt = 0.1 d, 1,000 steps, FP32 ages, the step loop replayed as CUDA
Graphs of 50 steps): graph ingest from the CSR already resident in HBM,
state initialisation and the 1,000 fused steps, timed with CUDA events on the
launching stream. The L2 is flushed between benchmark steps. The same metric
is also measured end to end through the C ABI with host buffers (pinned
CSR upload, counts download), and for the Barabasi-Albert (m = 5) graph of
the same size as a secondary figure.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl flashstep|reference]
Under torchrun every rank runs an independent replica (no data-path
collective): "replicas only" scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "GNUPS at N=1e6 (regular/BA); served-ensemble GNUPS + p50/p99 vs plain"
UNIT = "GNUPS"
# per step kernel: the committed ncu summary holding its DRAM traffic, and the
# sources whose hash must match for that traffic to be reported
PROFILE_TRAFFIC = {
    "push_step_kernel": os.path.join(ROOT, "profiles", "push_step_kernel_regular_n1e6.md"),
    "sell_smem_kernel": os.path.join(ROOT, "profiles", "sell_smem_kernel_regular_n1e6.md"),
}
KERNEL_SOURCES = {
    "push_step_kernel": ["paper_2604_22092_gb300/csrc/fs_push.cu", "paper_2604_22092_gb300/csrc/fs_device.cuh",
                         "paper_2604_22092_gb300/csrc/fs_internal.h"],
    "sell_smem_kernel": ["paper_2604_22092_gb300/csrc/fs_step.cu", "paper_2604_22092_gb300/csrc/fs_device.cuh",
                         "paper_2604_22092_gb300/csrc/fs_internal.h"],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["flashstep", "reference"], default="flashstep")
    ap.add_argument("--n", type=int, default=1_000_000, help="nodes (the headline workload uses 10^6)")
    ap.add_argument("--sim-steps", type=int, default=1000)
    ap.add_argument("--graph-steps", type=int, default=50)
    ap.add_argument("--no-secondary", action="store_true", help="skip the Barabasi-Albert figure")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true", help="skip the served-vs-plain block")
    ap.add_argument("--no-large", action="store_true", help="skip the N=1e8 block")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-graph packed-ensemble block")
    ap.add_argument("--workload", choices=["regular", "ensemble", "serving", "large", "precision", "shedding",
                                           "compaction", "markov"],
                    default="regular",
                    help="regular: the headline line; ensemble / serving: full-size packed and served runs; "
                         "shedding: constant vs age-dependent infectivity on regular d=8 and BA m=4 graphs; "
                         "compaction: runs with and without the active-node list on ER d=8 and BA m=4; "
                         "markov: the Markovian engine's transitions per second on ER d=8 (SIS, SIR)")
    ap.add_argument("--age", choices=["f32", "f16"], default="f32", help="age storage of ensemble/serving runs")
    ap.add_argument("--ens-graphs", type=int, default=64, help="graphs of the packed-ensemble run")
    ap.add_argument("--ens-steps", type=int, default=500, help="steps of the packed-ensemble run")
    ap.add_argument("--serve-requests", type=int, default=60, help="requests of --workload serving")
    ap.add_argument("--no-other-form", action="store_true", help="skip timing the other pressure form")
    ap.add_argument("--large-n", type=str, default="",
                    help="comma-separated N of --workload large (default: 1e7 and 1e8 FP32, 1e8 BF16)")
    ap.add_argument("--pressure", choices=["auto", "gather", "push"], default="auto",
                    help="pressure form of single-realisation runs (auto = push where available)")
    return ap.parse_args()


PRESSURE = {"auto": 0, "gather": 1, "push": 2}


# ------------------------------------------------------------------ workload
def workload(kind: str, n: int):
    if kind == "regular":
        g = W.random_regular(n, 10, seed=0)
        idx = W.index_nodes(g.n, 100, seed=1)
        name = f"seir-regular10-n{n:.0e}".replace("+0", "")
    else:
        g = W.barabasi_albert(n, 5, seed=0)
        idx = W.index_nodes(g.n, 100, seed=1, allowed=W.non_hub_nodes(g))
        name = f"seir-ba-m5-n{n:.0e}".replace("+0", "")
    return g, idx, name


def params(fs, seed: int, replicate: int = 0, pressure: int = 0):
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed,
                         latent=fs.law("weibull", 2.0, 4.0), replicate=replicate, pressure=pressure)


def push_bytes_model(counts: np.ndarray, n: int, d: int, b_age: int = 4) -> np.ndarray:
    """Algorithmic bytes of each step of the push formulation on a d-regular
    SEIR run, from its counts trajectory ((K+1) x 4, row k = state at the start
    of step k): every node's state is read (1 B); every S node reads its count
    and pending tally (1 + 2 B); every E/I node reads and writes its age
    (2 b_age); every transition writes a state byte; every node entering or
    leaving I reads its transposed row bounds (16 B) and, per out-edge, one
    column (4 B) and one tally read-modify-write (4 B)."""
    c = counts.astype(np.int64)
    S, E, I, R = c[:-1, 0], c[:-1, 1], c[:-1, 2], c[:-1, 3]
    left_s = S - c[1:, 0]
    to_r = c[1:, 3] - R
    enter_i = (c[1:, 2] - I) + to_r
    pushers = enter_i + to_r
    return (n * 1.0 + 3.0 * S + 2.0 * b_age * (E + I) + (left_s + enter_i + to_r)
            + pushers * (16.0 + d * 8.0))


def breq_regular(counts: np.ndarray, n: int, d: float, b_age: int = 4) -> float:
    """B_req (the pull formulation's required bytes, bytes_model) of the steps
    whose start states are rows 0 .. K-1 of a (K+1) x 4 counts trajectory on a
    d-regular graph, where every S node's row holds d edges."""
    S = counts[:-1, 0].astype(np.float64)
    return bytes_model(n, S.size, float(S.sum()), float(d * S.sum()), b_age=b_age)


def bytes_model(n: int, steps: int, s_node_sum: int, s_degree_sum: int, b_state=1, b_age=4) -> float:
    """Algorithmic bytes of `steps` steps of the pull formulation: every node
    reads and writes its state and age and writes its bitmap bit; every S node
    reads its row offset (4 B), and per in-edge a column index (4 B) and one
    bitmap bit."""
    return (n * steps * (2 * b_state + 2 * b_age + 1 / 8) + 4.0 * s_node_sum
            + (4.0 + 1 / 8) * s_degree_sum)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    try:
        text = open(PROFILE_TRAFFIC[kernel]).read()
    except (OSError, KeyError):
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    k = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not k or k.group(1) != kernel_source_hash(kernel):
        return None
    return float(m.group(1))


def step_kernel_name(fs, g, pressure: int) -> str:
    """The step kernel a sim runs: the push kernel for the push form; for the
    gather, the shared-memory-bitmap SELL kernel when the bitmap fits in
    shared memory, else the fused kernel."""
    if pressure == fs.FS_PRESSURE_PUSH:
        return "push_step_kernel"
    bm_bytes = (((g.n >> 5) + 1) * 4 + 15) // 16 * 16
    return "sell_smem_kernel" if bm_bytes <= 200 * 1024 else "fused_step_kernel"


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ the oracle on the host cores
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _host_worker(path: str, rep: int, conn) -> None:
    """One host core (a spawned process): the single-threaded oracle, as it
    stands, on one realisation (replicate `rep`) of the SEIR workload on the
    graph saved under `path`, advanced on command."""
    import oracle as om
    rp = np.load(path + "_rp.npy", mmap_mode="r")
    ci = np.load(path + "_ci.npy", mmap_mode="r")
    idx = np.load(path + "_idx.npy")
    prm = om.params(om.SEIR, om.law("weibull", 2.0, 4.0), om.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1,
                    seed=1, rep=rep)
    X, A = om.init(rp.size - 1, idx, om.E)
    k = 0
    conn.send("ready")
    while True:
        cmd = conn.recv()
        if cmd[0] == "stop":
            break
        if cmd[0] == "counts":
            conn.send((k, om.counts(X).tolist()))
            continue
        t0 = time.perf_counter()
        done = 0
        while done < cmd[1] and (cmd[0] == "steps" or time.perf_counter() - t0 < cmd[2]):
            X, A, _, _ = om.step(rp, ci, prm, k, X, A)
            k += 1
            done += 1
        conn.send((done, time.perf_counter() - t0))


class HostOracle:
    """The oracle run on every host core at once: one process per core, each
    stepping its own realisation (replicate index = worker number) of the same
    workload. Processes are spawned (never forked after CUDA has started)."""

    def __init__(self, g, idx, workers: int | None = None):
        import multiprocessing as mp
        import tempfile
        import oracle as om
        om.build()
        self.n = g.n
        self.tmp = tempfile.mkdtemp(prefix="fs_host_oracle_")
        path = os.path.join(self.tmp, "g")
        np.save(path + "_rp.npy", np.ascontiguousarray(g.row_ptr, dtype=np.int64))
        np.save(path + "_ci.npy", np.ascontiguousarray(g.col_ind, dtype=np.int32))
        np.save(path + "_idx.npy", np.ascontiguousarray(idx, dtype=np.int32))
        ctx = mp.get_context("spawn")
        self.workers = workers or host_cores()
        self.procs, self.conns = [], []
        for r in range(self.workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_host_worker, args=(path, r, b), daemon=True)
            p.start()
            self.procs.append(p)
            self.conns.append(a)
        for c in self.conns:
            assert c.recv() == "ready"

    def advance(self, steps: int, budget_s: float | None = None):
        """Every worker runs `steps` steps (or until `budget_s` passes); returns
        (node updates, wall seconds from the first command to the last reply)."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(("steps", steps) if budget_s is None else ("run", steps, budget_s))
        done = [c.recv() for c in self.conns]
        wall = time.perf_counter() - t0
        return self.n * sum(d for d, _ in done), wall, [d for d, _ in done]

    def counts(self):
        """(steps run, compartment counts) of every worker's realisation."""
        for c in self.conns:
            c.send(("counts",))
        return [c.recv() for c in self.conns]

    def close(self):
        import shutil
        for c in self.conns:
            c.send(("stop",))
        for p in self.procs:
            p.join(timeout=30)
        shutil.rmtree(self.tmp, ignore_errors=True)


def cpu_baseline(graphs, budget_s=10.0, max_steps=400):
    """The oracle, as it stands, on every host core (one independent
    realisation per core) over the first steps of each workload from its
    initial state. `graphs`: [(name, graph, index nodes)]; the first is the
    headline workload."""
    out = None
    for name, g, idx in graphs:
        h = HostOracle(g, idx)
        try:
            upd, wall, steps = h.advance(max_steps, budget_s)
        finally:
            h.close()
        r = {"value": upd / wall / 1e9, "unit": UNIT, "cores": h.workers, "kind": "oracle",
             "sample": f"{name}: {h.workers} processes, one per host core, each the single-threaded C oracle on "
                       f"its own realisation (replicates 0..{h.workers - 1}) from the initial state for "
                       f"{min(steps)}-{max(steps)} steps (first {budget_s:.0f} s)",
             "seconds": round(wall, 3), "workload": name}
        if out is None:
            out = r
        else:
            out.setdefault("other", []).append(r)
    return out


# ------------------------------------------------------------------ ensembles and serving
def scen_params(fs, sc, replicate: int, age_dtype: int, pressure: int = 0, seed: int | None = None):
    """One scenario's parameters. The realisations of a request draw from one
    Philox key (the request's seed) and are told apart by the replicate index
    (scenario * replicates + replicate)."""
    latent = fs.law("erlang", 0.75, k=3) if sc.latent == "erlang" else fs.law("weibull", 2.0, 4.0)
    return fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), float(sc.sigma_inf)), float(sc.beta), 0.1,
                         int(sc.seed if seed is None else seed), latent=latent, replicate=replicate,
                         age_dtype=age_dtype, pressure=pressure)


def index_for(g, count=100, seed=1):
    allowed = W.non_hub_nodes(g) if g.name.startswith("ba") else None
    pool = g.n if allowed is None else allowed.size
    return W.index_nodes(g.n, min(count, max(1, pool // 2)), seed=seed, allowed=allowed)


def plain_seconds(fs, gh, p, idx, steps):
    """One realisation through the one-run-per-launch engine, wall time."""
    t0 = time.perf_counter()
    s = fs.fs_sim_init(gh, p, idx)
    fs.fs_sim_run(s, steps, 50, want_counts=True)
    fs.fs_sim_destroy(s)
    return time.perf_counter() - t0


def _gen_mixed(job):
    """One graph of the mixed family, written to .npy files (a spawned worker)."""
    q, n_lo, n_hi, seed, path = job
    g = W.mixed_graph(q, n_lo, n_hi, seed=seed)
    np.save(os.path.join(path, f"rp{q}.npy"), g.row_ptr)
    np.save(os.path.join(path, f"ci{q}.npy"), g.col_ind)
    return q, g.n, g.name


def mixed_graphs(n_graphs: int, n_lo: float, n_hi: float, seed: int):
    """The mixed graph family (workloads.mixed_graph), generated on every host
    core at once by spawned workers (the same graphs as a serial loop)."""
    import multiprocessing as mp
    import shutil
    import tempfile
    tmp = tempfile.mkdtemp(prefix="fs_mixed_")
    try:
        with mp.get_context("spawn").Pool(max(1, min(host_cores(), n_graphs))) as pool:
            done = pool.map(_gen_mixed, [(q, n_lo, n_hi, seed, tmp) for q in range(n_graphs)], chunksize=1)
        graphs = []
        for q, n, name in sorted(done):
            graphs.append(W.Graph(n, np.load(os.path.join(tmp, f"rp{q}.npy")),
                                  np.load(os.path.join(tmp, f"ci{q}.npy")), name))
        return graphs
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def ensemble_bench(fs, torch, n_graphs, n_lo, n_hi, steps, age_dtype, reps=3, pressure=0, graphs=None):
    """Packed batch of 8 scenarios x n_graphs mixed graphs in one launch per
    step, against every one of those realisations run alone through the plain
    one-run-per-launch engine (fs_sim_run, CUDA Graph step loop), back to back."""
    if graphs is None:
        graphs = mixed_graphs(n_graphs, n_lo, n_hi, seed=2026)
    ghs = [fs.fs_graph_create(g.n, g.row_ptr, g.col_ind) for g in graphs]
    idxs = [index_for(g, seed=q + 1) for q, g in enumerate(graphs)]
    scen = [W.scenarios(8, seed=1000 + q) for q in range(n_graphs)]
    req_seed = [int(sc[0].seed) for sc in scen]          # each graph's 8 scenarios are one request
    stream = torch.cuda.Stream()
    times = []
    for it in range(reps):
        ens = [fs.fs_ens_create(ghs[q], [scen_params(fs, sc, s, age_dtype, pressure, seed=req_seed[q])
                                         for s, sc in enumerate(scen[q])], idxs[q])
               for q in range(n_graphs)]
        b = fs.fs_batch_create(age_dtype, n_graphs + 1, stream=stream)
        for e in ens:
            fs.fs_batch_add(b, e, steps)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        fs.fs_batch_run(b, steps + 1, 50)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) * 1e-3)
        fs.fs_batch_destroy(b)
        for e in ens:
            fs.fs_ens_destroy(e)
    served_s = float(np.median(times))
    updates = sum(g.n for g in graphs) * 8 * steps
    # the plain engine: every realisation alone, one after the other (a first
    # pass over scenario 0 of each graph warms the step code and the caches)
    for q in range(n_graphs):
        plain_seconds(fs, ghs[q], scen_params(fs, scen[q][0], 0, age_dtype, seed=req_seed[q]), idxs[q], steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(n_graphs):
        for s_, sc in enumerate(scen[q]):
            plain_seconds(fs, ghs[q], scen_params(fs, sc, s_, age_dtype, seed=req_seed[q]), idxs[q], steps)
    plain_s = time.perf_counter() - t0
    # the same, in the paper's one-run-per-launch form (Algorithm 3's gather
    # of the infectious neighbours every step)
    for q in range(n_graphs):
        plain_seconds(fs, ghs[q], scen_params(fs, scen[q][0], 0, age_dtype, fs.FS_PRESSURE_GATHER, seed=req_seed[q]),
                      idxs[q], steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(n_graphs):
        for s_, sc in enumerate(scen[q]):
            plain_seconds(fs, ghs[q], scen_params(fs, sc, s_, age_dtype, fs.FS_PRESSURE_GATHER, seed=req_seed[q]),
                          idxs[q], steps)
    plain_gather_s = time.perf_counter() - t0
    for gh in ghs:
        fs.fs_graph_destroy(gh)
    return {"workload": f"packed-{n_graphs}graphs-x8scen-n{n_lo:.0e}-{n_hi:.0e}-{steps}steps".replace("+0", ""),
            "realisations": 8 * n_graphs, "nodes_total": int(sum(g.n for g in graphs)),
            "age_storage": "f16" if age_dtype == fs.FS_AGE_F16 else "f32",
            "served_gnups": round(updates / served_s / 1e9, 3), "served_seconds": round(served_s, 4),
            "plain_gnups": round(updates / plain_s / 1e9, 3), "plain_seconds": round(plain_s, 3),
            "speedup": round(plain_s / served_s, 2),
            "plain_gather_gnups": round(updates / plain_gather_s / 1e9, 3),
            "plain_gather_seconds": round(plain_gather_s, 3),
            "speedup_vs_gather": round(plain_gather_s / served_s, 2),
            "plain_engine": "every realisation run alone through fs_sim_run (init + CUDA Graph step loop + "
                            "counts read back), back to back, host wall clock; plain_*: the library's default "
                            "single-realisation form (infection counts kept by pushes); plain_gather_*: the "
                            "paper's form (Algorithm 3, every S node gathers its row each step)",
            "request_seeds": "one Philox key per graph (its 8 scenarios are one request), replicate index = "
                             "scenario number"}


def serving_bench(fs, torch, n_requests, n_pool, n_hi, steps, rep_lo, rep_hi, window_s, age_dtype, big_n=0,
                  big_age=None, plain_sample=0):
    """A Poisson stream of requests against the server (optionally beside one
    big SEIR job on a random 10-regular graph of big_n nodes, run on its own
    stream at the same time), then the same stream through the plain engine:
    every request's realisations alone through fs_sim_run, one request after
    the other in arrival order. The plain service time of a request is the
    sum of the measured run times of all its realisations (plain_sample = 0)
    or the mean over a random sample of plain_sample of them times its
    realisation count; the plain queue (and the big job, run alone after it)
    is replayed on those measured times against the arrival times."""
    pool = mixed_graphs(n_pool, 1e4, n_hi, seed=77)
    ghs = [fs.fs_graph_create(g.n, g.row_ptr, g.col_ind) for g in pool]
    idxs = [index_for(g, seed=q + 5) for q, g in enumerate(pool)]
    reqs = W.request_stream(n_requests, n_requests / window_s, n_pool, seed=99, steps=steps, rep_lo=rep_lo,
                            rep_hi=rep_hi)
    srv = fs.fs_server_create(quantum=10, age_dtype=age_dtype)
    # warm the server's graph capture on a tiny request
    wid = fs.fs_server_submit(srv, ghs[0], [scen_params(fs, W.scenarios(1, 5)[0], 0, age_dtype)], 1, idxs[0], 5)
    fs.fs_server_drain(srv, 120)
    big = None
    if big_n:
        dev = torch.device("cuda")
        rp, col = device_regular(torch, int(big_n), 10, seed=0, dev=dev)
        bstream = torch.cuda.Stream()
        bgh = fs.fs_graph_create(int(big_n), rp, col, opts=fs.graph_opts(device_input=True), stream=bstream)
        bprm = fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, 1,
                             latent=fs.law("weibull", 2.0, 4.0), age_dtype=big_age if big_age is not None else age_dtype)
        bidx = W.index_nodes(int(big_n), 100, seed=1)
        # alone first (its plain time), then beside the request stream
        t_b = time.perf_counter()
        bsh = fs.fs_sim_init(bgh, bprm, bidx, stream=bstream)
        fs.fs_sim_run(bsh, 1000, 50, want_counts=False)
        big_alone = time.perf_counter() - t_b
        fs.fs_sim_destroy(bsh)
        bsh = fs.fs_sim_init(bgh, bprm, bidx, stream=bstream)
        big = {"n": int(big_n), "steps": 1000, "alone_s": round(big_alone, 3)}
    t0 = time.perf_counter()
    if big:
        fs.fs_sim_run_async(bsh, 1000, 50)
    ids = []
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival:
            time.sleep(0.0002)
        sc = W.scenarios(r.n_scen, seed=r.seed)
        ids.append(fs.fs_server_submit(srv, ghs[r.graph],
                                       [scen_params(fs, c, j * r.replicates, age_dtype, seed=r.seed)
                                        for j, c in enumerate(sc)], r.replicates, idxs[r.graph], r.steps))
    fs.fs_server_drain(srv, 3600)
    stream_done = time.perf_counter() - t0
    if big:
        fs.fs_sim_sync(bsh)
    makespan = time.perf_counter() - t0
    lat = np.array([fs.fs_server_poll(srv, rid)[2] for rid in ids])
    fs.fs_server_destroy(srv)
    updates = sum(pool[r.graph].n * r.n_scen * r.replicates * r.steps for r in reqs)
    big_updates = 0
    if big:
        big["counts_final"] = [int(x) for x in fs.fs_sim_run(bsh, 0)[0]]
        fs.fs_sim_destroy(bsh)
        fs.fs_graph_destroy(bgh)
        big_updates = big["n"] * big["steps"]
    # the plain engine: a random sample of each request's realisations, each
    # alone (a warm-up run first for every graph)
    rng = np.random.default_rng(2027)
    for q in range(n_pool):
        plain_seconds(fs, ghs[q], scen_params(fs, W.scenarios(1, seed=q)[0], 0, age_dtype), idxs[q], 5)
    clock, plain_lat, sampled = 0.0, [], 0
    for r in reqs:
        sc = W.scenarios(r.n_scen, seed=r.seed)
        total = r.n_scen * r.replicates
        every = plain_sample <= 0 or plain_sample >= total
        picks = np.arange(total) if every else rng.choice(total, size=plain_sample, replace=False)
        secs = []
        for pk in picks:
            j, rep = int(pk) // r.replicates, int(pk) % r.replicates
            p = scen_params(fs, sc[j], j * r.replicates + rep, age_dtype, seed=r.seed)
            secs.append(plain_seconds(fs, ghs[r.graph], p, idxs[r.graph], r.steps))
        sampled += len(secs)
        service = float(np.sum(secs)) if every else float(np.mean(secs)) * total
        start = max(clock, r.arrival)
        clock = start + service
        plain_lat.append(clock - r.arrival)
    plain_lat = np.array(plain_lat)
    plain_total = clock + (big["alone_s"] if big else 0.0)
    for gh in ghs:
        fs.fs_graph_destroy(gh)
    out = {"workload": f"serving-{n_requests}req-pool{n_pool}-n1e4-{n_hi:.0e}-{steps}steps-rep{rep_lo}-{rep_hi}".replace("+0", "")
                       + (f"+seir-regular10-n{big_n:.0e}".replace("+0", "") if big else ""),
           "arrival_rate_per_s": round(n_requests / window_s, 2),
           "served_gnups": round((updates + big_updates) / makespan / 1e9, 3), "served_makespan_s": round(makespan, 3),
           "served_stream_s": round(stream_done, 3),
           "served_p50_s": round(float(np.percentile(lat, 50)), 4), "served_p99_s": round(float(np.percentile(lat, 99)), 4),
           "plain_gnups": round((updates + big_updates) / plain_total / 1e9, 3), "plain_makespan_s": round(plain_total, 3),
           "plain_p50_s": round(float(np.percentile(plain_lat, 50)), 4),
           "plain_p99_s": round(float(np.percentile(plain_lat, 99)), 4),
           "speedup": round(plain_total / makespan, 2), "node_updates": int(updates + big_updates),
           "plain_engine": (f"every realisation of every request run alone through fs_sim_run ({sampled} runs), "
                            f"each request's service time their sum"
                            if plain_sample <= 0 else
                            f"every request's service time measured on a random sample of its realisations "
                            f"({sampled} runs in all, each alone through fs_sim_run), scaled by its realisation "
                            f"count")
                           + "; requests one after the other in arrival order, queue replayed on those times"
                           + ("; the big job run alone after them" if big else "")}
    if big:
        big["age_storage"] = {fs.FS_AGE_F32: "f32", fs.FS_AGE_F16: "f16", fs.FS_AGE_BF16: "bf16"}[bprm.age_dtype]
        out["big_job"] = big
    return out


# ------------------------------------------------------------------ arms
def run_flashstep(args, rank, world, local_rank):
    import torch
    import paper_2604_22092_gb300 as fs
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    fs.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    g, idx, wname = workload("regular", args.n)
    stream = torch.cuda.Stream(device=dev)
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col_ind).to(dev)
    counts_dev = torch.zeros((args.sim_steps + 1) * 4, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prm = params(fs, seed=replica_seed(rank), replicate=0, pressure=PRESSURE[args.pressure])
    opts = fs.graph_opts(device_input=True)

    def one_step(prm_run):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gh = fs.fs_graph_create(g.n, d_rp, d_col, opts=opts, stream=stream)
        sh = fs.fs_sim_init(gh, prm_run, idx, stream=stream)
        replay_ms = fs.fs_sim_run_timed(sh, args.sim_steps, args.graph_steps, counts_dev)
        ev1.record(stream)
        ev1.synchronize()
        work = fs.fs_sim_work(sh)
        work["pressure"] = fs.fs_sim_pressure_get(sh)
        fs.fs_sim_destroy(sh)
        fs.fs_graph_destroy(gh)
        return ev0.elapsed_time(ev1), replay_ms, work

    K = args.graph_steps
    full = args.sim_steps // K
    steps_in_graphs = full * K

    def step_bytes(work, pressure):
        """Algorithmic bytes of the steps inside the timed graph replays, in the
        byte model of the form that ran."""
        if pressure == fs.FS_PRESSURE_PUSH:
            cnt = counts_dev.view(args.sim_steps + 1, 4).cpu().numpy()
            return float(np.sum(push_bytes_model(cnt, g.n, 10)[:steps_in_graphs]))
        return (bytes_model(g.n, args.sim_steps, work["s_node_sum"], work["s_degree_sum"])
                * steps_in_graphs / args.sim_steps)

    def breq_of_run():
        cnt = counts_dev.view(args.sim_steps + 1, 4).cpu().numpy()
        return breq_regular(cnt[:steps_in_graphs + 1], g.n, g.col_ind.size / g.n)

    def roofline_of(bytes_per_step, step_ms, kernel, pressure, breq_per_step=None):
        peak, peak_kind = measured_peak_hbm()
        achieved = bytes_per_step / (step_ms * 1e-3) / 1e9
        # the paper's dense traffic model (every row traversed): N (2 b_s + 2 b_a + 1/8 + 4) + E (4 + 1/8)
        dense_bytes = g.n * (2 + 8 + 1 / 8 + 4) + g.col_ind.size * (4 + 1 / 8)
        model = ("push: state read by every node, count + pending tally by S nodes, ages by E/I nodes, "
                 "state writes, transposed row bounds + 8 B per out-edge of nodes entering or leaving I"
                 if pressure == fs.FS_PRESSURE_PUSH else
                 "gather: state/age read+write and bitmap bit per node, row offset per S node, "
                 "column + bitmap bit per S-row edge")
        extra = {}
        if breq_per_step is not None:
            # the same trajectory's B_req (the gather's required bytes) over the
            # push step's time: the byte figure the two forms share
            extra = {"breq_equiv_frac": round(breq_per_step / (step_ms * 1e-3) / 1e9 / peak, 4),
                     "breq_bytes_per_step": round(breq_per_step)}
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": profiled_traffic(kernel), **extra,
                "peak_source": peak_kind, "kernel": kernel,
                "algorithmic_bytes_per_launch": round(bytes_per_step), "byte_model": model,
                "avg_launch_us": round(step_ms * 1e3, 3),
                "dense_equiv_frac": round(dense_bytes / (step_ms * 1e-3) / 1e9 / peak, 4),
                "note": "at N=1e6 the step's working set is L2-resident across steps, so the step is "
                        "latency-bound; the HBM-bound N=1e7/1e8 points are bench.py --workload large"}

    # the clock sampler starts before the warm-up, so that its own start-up
    # (nvidia-smi loading NVML) does not fall into the timed steps
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        one_step(prm)
    torch.cuda.synchronize()
    times, kern_ms, bytes_alg, breq_alg = [], [], [], []
    pressure_used = None
    launches0 = fs.fs_kernel_launches()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms, replay_ms, work = one_step(prm)
        torch.cuda.synchronize()
        times.append(ms)
        kern_ms.append(float(np.sum(replay_ms[:full])))
        pressure_used = work["pressure"]
        bytes_alg.append(step_bytes(work, pressure_used))
        if pressure_used == fs.FS_PRESSURE_PUSH:
            breq_alg.append(breq_of_run())
    clock_info = clocks.stop() if clocks else None
    # the library's kernel launches inside the timed region (all K benchmark
    # steps; graph replays count their kernel nodes), and per benchmark step
    launches_total = fs.fs_kernel_launches() - launches0
    launches = launches_total // max(args.steps, 1)
    total_ms = max_over_ranks(float(np.sum(times)), dist, dev)
    value = whole_job_gnups(g.n, args.sim_steps, args.steps, world, total_ms)
    # roofline of the dominant kernel (the step): algorithmic bytes of the
    # steps / their event-timed graph replays (which include launch gaps and the
    # per-replay epilogue, so this is a lower bound on the kernel's own rate)
    per_step_bytes = float(np.sum(bytes_alg)) / (args.steps * steps_in_graphs)
    per_step_ms = float(np.sum(kern_ms)) / (args.steps * steps_in_graphs)
    kernel = step_kernel_name(fs, g, pressure_used)
    roofline = roofline_of(per_step_bytes, per_step_ms, kernel, pressure_used,
                           float(np.sum(breq_alg)) / (args.steps * steps_in_graphs) if breq_alg else None)
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wname, "model": "SEIR renewal", "graph": "random 10-regular (configuration model, seed 0)",
                      "n": g.n, "sim_steps": args.sim_steps, "graph_steps": args.graph_steps,
                      "age_storage": "f32", "state_storage": "u8", "parallelism": f"replicas{world}",
                      "pressure": "push" if pressure_used == fs.FS_PRESSURE_PUSH else "gather",
                      "l2_flush": "512 MB write between timed steps",
                      "timed": "device-resident CSR -> ingest + init + all steps (CUDA events)"},
           "roofline": roofline, "gpu_launches": int(launches_total),
           "gpu_launches_per_step": int(launches)}
    if clock_info:
        out["clocks"] = clock_info
    # the other pressure form on the same workload (rank 0; not part of the timed value)
    if rank == 0 and not args.no_other_form:
        other = fs.FS_PRESSURE_GATHER if pressure_used == fs.FS_PRESSURE_PUSH else fs.FS_PRESSURE_PUSH
        prm_o = params(fs, seed=replica_seed(rank), replicate=0, pressure=other)
        one_step(prm_o)
        o_times, o_kern, o_bytes = [], [], []
        for _ in range(2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ms, replay_ms, work = one_step(prm_o)
            o_times.append(ms)
            o_kern.append(float(np.sum(replay_ms[:full])))
            o_bytes.append(step_bytes(work, work["pressure"]))
        o_ms = float(np.mean(o_times))
        out["other_form"] = {
            "pressure": "push" if other == fs.FS_PRESSURE_PUSH else "gather",
            "value": round(g.n * args.sim_steps / (o_ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "ms_per_step": round(o_ms, 3),
            "roofline": roofline_of(float(np.sum(o_bytes)) / (2 * steps_in_graphs),
                                    float(np.sum(o_kern)) / (2 * steps_in_graphs),
                                    step_kernel_name(fs, g, other), other)}
    # end to end through the C ABI with host buffers (rank 0 only)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e(fs, torch, g, idx, prm, args, stream)
    if rank == 0 and not args.no_secondary:
        out["secondary"] = secondary_ba(fs, torch, args, stream, flush)
    # the HBM-bound points: N = 10^8, FP32 and BF16 ages, whole job (rank 0)
    if rank == 0 and not args.no_large:
        out["large"] = []
        for a in (fs.FS_AGE_F32, fs.FS_AGE_BF16):
            cs = ClockSampler(local_rank)
            cs.start()
            r = large_bench(fs, torch, 100_000_000, a, args.sim_steps, args.graph_steps, reps=1,
                            pressure=PRESSURE[args.pressure])
            r.pop("phases_step_us_gbs_sfrac", None)
            r["clocks"] = cs.stop()
            out["large"].append(r)
    # the 64-graph x 8-scenario packed ensemble against every realisation run
    # alone, FP32 and FP16 ages (rank 0)
    if rank == 0 and not args.no_ensemble:
        graphs = mixed_graphs(args.ens_graphs, 1e4, 2e6, seed=2026)
        out["ensemble"] = []
        for a in (fs.FS_AGE_F32, fs.FS_AGE_F16):
            cs = ClockSampler(local_rank)
            cs.start()
            r = ensemble_bench(fs, torch, n_graphs=args.ens_graphs, n_lo=1e4, n_hi=2e6, steps=args.ens_steps,
                               age_dtype=a, graphs=graphs)
            r["clocks"] = cs.stop()
            out["ensemble"].append(r)
        del graphs
    if rank == 0 and not args.no_served:
        out["served"] = serving_bench(fs, torch, n_requests=24, n_pool=8, n_hi=2e5, steps=200, rep_lo=16,
                                      rep_hi=64, window_s=0.25, age_dtype=fs.FS_AGE_F32)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        gb, ib, nb = workload("ba", args.n)
        out["cpu_baseline"] = cpu_baseline([(wname, g, idx), (nb, gb, ib)])
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out if rank == 0 else None


def e2e(fs, torch, g, idx, prm, args, stream):
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col_ind).pin_memory()
    idx_h = np.ascontiguousarray(idx, dtype=np.int32)
    times = []
    for it in range(args.warmup + args.steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gh = fs.fs_graph_create(g.n, rp_h.data_ptr(), col_h.data_ptr(), stream=stream)
        sh = fs.fs_sim_init(gh, prm, idx_h, stream=stream)
        counts = fs.fs_sim_run(sh, args.sim_steps, args.graph_steps)
        ev1.record(stream)
        ev1.synchronize()
        if it >= args.warmup:
            times.append(ev0.elapsed_time(ev1))
        fs.fs_sim_destroy(sh)
        fs.fs_graph_destroy(gh)
    assert counts.sum(axis=1).max() == g.n
    ms = float(np.mean(times))
    return {"value": round(g.n * args.sim_steps / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col_ind.nbytes + idx_h.nbytes),
            "d2h_bytes_per_step": int((args.sim_steps + 1) * 16), "ms_per_step": round(ms, 3)}


def secondary_ba(fs, torch, args, stream, flush):
    g, idx, wname = workload("ba", args.n)
    dev = flush.device
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col_ind).to(dev)
    prm = params(fs, seed=1, pressure=PRESSURE[args.pressure])
    # the class split is chosen by the autotuner (its trials run once, in the
    # first warm-up creation; later creations are answered from its cache)
    opts = fs.graph_opts(dispatch=fs.FS_DISPATCH_TUNE, device_input=True)
    times = []
    info = None
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gh = fs.fs_graph_create(g.n, d_rp, d_col, opts=opts, stream=stream)
        sh = fs.fs_sim_init(gh, prm, idx, stream=stream)
        fs.fs_sim_run_async(sh, args.sim_steps, args.graph_steps)
        fs.fs_sim_sync(sh)
        ev1.record(stream)
        ev1.synchronize()
        if it >= args.warmup:
            times.append(ev0.elapsed_time(ev1))
        info = fs.fs_graph_info_get(gh)
        fs.fs_sim_destroy(sh)
        fs.fs_graph_destroy(gh)
    ms = float(np.mean(times))
    return {"workload": wname, "value": round(g.n * args.sim_steps / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "ms_per_step": round(ms, 3), "d_max": info["d_max"], "rho": round(info["rho"], 1),
            "thread_class_nodes": info["n_thread"], "merge_class_nodes": info["n_merge"],
            "dispatch": f"tuned: thread_max_deg {info['thread_max_deg']}"}


def device_regular(torch, n: int, d: int, seed: int, dev):
    """Random d-regular multigraph built on the device for N too large for the
    host generator: configuration-model stub pairing by a seeded device
    permutation. Node i owns stubs i*d .. i*d + d - 1, so each stub's column is
    its partner's node and the CSR needs no sort. Self-loops and repeated edges
    (about (d-1)/2 + (d-1)^2/4 expected in the whole graph) are kept."""
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    perm = torch.randperm(n * d, generator=gen, device=dev)
    a, b = perm[0::2], perm[1::2]
    col = torch.empty(n * d, dtype=torch.int32, device=dev)
    col[a] = torch.div(b, d, rounding_mode="floor").to(torch.int32)
    col[b] = torch.div(a, d, rounding_mode="floor").to(torch.int32)
    del perm, a, b
    rp = torch.arange(0, (n + 1) * d, d, dtype=torch.int64, device=dev)
    return rp, col


def large_bench(fs, torch, n: int, age_dtype: int, sim_steps: int, graph_steps: int, reps: int, pressure: int = 0):
    """The C1 SEIR workload on a random 10-regular graph of N = 10^7 or 10^8
    nodes, where the step's working set is far larger than L2: ingest from the
    device CSR + init + all steps, timed with CUDA events; the kernel-side
    roofline uses the graph replays alone."""
    dev = torch.device("cuda")
    d = 10
    rp, col = device_regular(torch, n, d, seed=0, dev=dev)
    idx = W.index_nodes(n, 100, seed=1)
    prm = fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, 1,
                        latent=fs.law("weibull", 2.0, 4.0), replicate=0, age_dtype=age_dtype, pressure=pressure)
    opts = fs.graph_opts(device_input=True)
    stream = torch.cuda.Stream()
    b_age = 4 if age_dtype == fs.FS_AGE_F32 else 2
    totals, replays, breq = [], [], []
    counts_dev = torch.zeros((sim_steps + 1) * 4, dtype=torch.int32, device=dev)
    for it in range(reps + 1):
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gh = fs.fs_graph_create(n, rp, col, opts=opts, stream=stream)
        sh = fs.fs_sim_init(gh, prm, idx, stream=stream)
        ms = fs.fs_sim_run_timed(sh, sim_steps, graph_steps, counts_dev)
        ev1.record(stream)
        ev1.synchronize()
        work = fs.fs_sim_work(sh)
        pressure_used = fs.fs_sim_pressure_get(sh)
        cnt = counts_dev.view(sim_steps + 1, 4).cpu().numpy().astype(np.int64)
        counts = fs.fs_sim_run(sh, 0)
        gbytes = fs.fs_graph_info_get(gh)["device_bytes"]
        fs.fs_sim_destroy(sh)
        fs.fs_graph_destroy(gh)
        if it == 0:
            continue                        # warm-up: graph capture, first-touch of the pools
        full = sim_steps // graph_steps
        totals.append(ev0.elapsed_time(ev1))
        replays.append(float(np.sum(ms[:full])))
        if pressure_used == fs.FS_PRESSURE_PUSH:
            step_b = push_bytes_model(cnt, n, d, b_age)
            breq.append(float(np.sum(step_b[:full * graph_steps])))
        else:
            step_b = None
            breq.append(bytes_model(n, sim_steps, work["s_node_sum"], work["s_degree_sum"], b_age=b_age)
                        * full * graph_steps / sim_steps)
    assert int(counts[-1].sum()) == n
    peak, peak_kind = measured_peak_hbm()
    # per replay of graph_steps steps: time per step and B_req rate (S-degree sum
    # = d x |S| on a d-regular graph)
    phases = []
    for r in range(sim_steps // graph_steps):
        S = cnt[r * graph_steps:(r + 1) * graph_steps, 0]
        if step_b is not None:
            b = float(np.sum(step_b[r * graph_steps:(r + 1) * graph_steps]))
        else:
            b = graph_steps * n * (2 + 2 * b_age + 1 / 8) + float(S.sum()) * (4 + d * (4 + 1 / 8))
        phases.append([r * graph_steps, round(float(ms[r]) * 1e3 / graph_steps, 1),
                       round(b / (float(ms[r]) * 1e-3) / 1e9, 0), round(float(S.mean()) / n, 3)])
    steps_timed = (sim_steps // graph_steps) * graph_steps
    step_ms = float(np.mean(replays)) / steps_timed
    per_step_bytes = float(np.mean(breq)) / steps_timed
    dense = n * (2 + 2 * b_age + 1 / 8 + 4) + n * d * (4 + 1 / 8)
    total_ms = float(np.mean(totals))
    return {"workload": f"seir-regular10-n{n:.0e}-{'f32' if b_age == 4 else 'bf16'}".replace("+0", ""),
            "n": n, "sim_steps": sim_steps, "age_storage": "f32" if b_age == 4 else "bf16",
            "value": round(n * sim_steps / (total_ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "ms_total": round(total_ms, 2), "steps_gnups": round(n / (step_ms * 1e-3) / 1e9, 3),
            "avg_step_us": round(step_ms * 1e3, 2),
            "roofline": {"bound": "hbm", "achieved": round(per_step_bytes / (step_ms * 1e-3) / 1e9, 1),
                         "peak": peak, "unit": "GB/s", "peak_source": peak_kind,
                         "frac": round(per_step_bytes / (step_ms * 1e-3) / 1e9 / peak, 4),
                         "frac_dense": round(dense / (step_ms * 1e-3) / 1e9 / peak, 4),
                         "algorithmic_bytes_per_step": round(per_step_bytes),
                         "dense_bytes_per_step": round(dense)},
            "pressure": "push" if pressure_used == fs.FS_PRESSURE_PUSH else "gather",
            "phases_step_us_gbs_sfrac": phases,
            "final_counts": [int(x) for x in counts[-1]], "graph_device_bytes": int(gbytes),
            "graph": "random 10-regular multigraph, device stub pairing (seed 0)"}


def precision_runs(fs, g, idx, model, inf, lat, beta, steps, reps, index_state=None):
    """Peak infectious fraction and attack rate of `reps` replicates under each
    age storage (one packed batch per storage type)."""
    n = g.n
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    peak, attack, secs = {}, {}, {}
    for name, a in (("f32", fs.FS_AGE_F32), ("f16", fs.FS_AGE_F16), ("bf16", fs.FS_AGE_BF16)):
        b = fs.fs_batch_create(a, (reps + 31) // 32 + 1)
        ens, outs = [], []
        for off in range(0, reps, 32):
            R = min(32, reps - off)
            prm = [fs.sim_params(model, inf, beta, 0.1, 1, latent=lat, replicate=off + q, age_dtype=a,
                                 index_state=index_state) for q in range(R)]
            e = fs.fs_ens_create(gh, prm, idx)
            o = np.zeros((steps + 1, R, 4), dtype=np.uint32)
            fs.fs_batch_add(b, e, steps, o)
            ens.append(e)
            outs.append(o)
        t0 = time.perf_counter()
        fs.fs_batch_run(b, steps + 1, 50)
        secs[name] = time.perf_counter() - t0
        fs.fs_batch_destroy(b)
        for e in ens:
            fs.fs_ens_destroy(e)
        c = np.concatenate(outs, axis=1).astype(np.int64)          # [steps+1, reps, 4]
        assert (c.sum(axis=2) == n).all()
        peak[name] = c[:, :, 2].max(axis=0) / n
        attack[name] = 1.0 - c[-1, :, 0] / n
    fs.fs_graph_destroy(gh)
    res = {}
    for name in ("f32", "f16", "bf16"):
        r = {"peak_I_mean": round(float(peak[name].mean()), 6), "attack_mean": round(float(attack[name].mean()), 6),
             "peak_I_sd": round(float(peak[name].std(ddof=1)), 6), "attack_sd": round(float(attack[name].std(ddof=1)), 6),
             "gnups": round(n * reps * steps / secs[name] / 1e9, 1)}
        if name != "f32":
            dp, da = peak[name] - peak["f32"], attack[name] - attack["f32"]
            r["peak_I_shift"] = float(f"{dp.mean():.3g}")
            r["peak_I_shift_se"] = float(f"{dp.std(ddof=1) / math.sqrt(reps):.3g}")
            r["attack_shift"] = float(f"{da.mean():.3g}")
            r["attack_shift_se"] = float(f"{da.std(ddof=1) / math.sqrt(reps):.3g}")
        res[name] = r
    return res


def precision_bench(fs, torch, n: int, steps: int, reps: int):
    """Storage precision of ages, stated per result. `reps` replicates of three
    workloads with FP32, FP16 and BF16 age storage: C1 (SEIR, 10-regular, N,
    beta 0.25, `steps` steps), the same at beta 0.05 (partial attack), and C0
    (SIR, 10-regular, N = 10^4, beta 0.3, log-normal(ln 5, 0.5), 10 index
    cases, 300 steps). Replicate r has the same random stream under every
    storage type, so the paired differences of each replicate's peak
    infectious fraction and attack rate isolate the effect of the storage. The
    FP32 trajectories are the oracle's (bit-exact parity), so the shifts are
    against the FP64 oracle at FP32 storage. Also the largest relative error of
    the GPU's FP32 hazards against FP64 closed forms over the ages a run visits."""
    import scipy.stats as st
    lat, inf = fs.law("weibull", 2.0, 4.0), fs.law("lognormal", math.log(6.0), 0.6)
    g = W.random_regular(n, 10, seed=0)
    idx = W.index_nodes(n, 100, seed=1)
    out = {"workload": f"age-storage-precision-{reps}replicates", "replicates": reps, "results": {}}
    out["results"][f"C1 seir-regular10-n{n:.0e} beta0.25 {steps}steps".replace("+0", "")] = \
        precision_runs(fs, g, idx, fs.FS_SEIR, inf, lat, 0.25, steps, reps)
    out["results"][f"C1 seir-regular10-n{n:.0e} beta0.05 {steps}steps".replace("+0", "")] = \
        precision_runs(fs, g, idx, fs.FS_SEIR, inf, lat, 0.05, steps, reps)
    g0 = W.random_regular(10_000, 10, seed=0)
    idx0 = W.index_nodes(g0.n, 10, seed=1)
    out["results"]["C0 sir-regular10-n1e4 beta0.3 300steps"] = \
        precision_runs(fs, g0, idx0, fs.FS_SIR, fs.law("lognormal", math.log(5.0), 0.5), None, 0.3, 300, reps)
    # GPU FP32 hazards against FP64 closed forms at the ages of the fixed-step sequence
    tau = (np.arange(1, 1001) * np.float32(0.1)).astype(np.float32)
    t64 = tau.astype(np.float64)
    refs = {"lognormal(ln 6, 0.6)": (inf, np.exp(st.lognorm.logpdf(t64, 0.6, scale=6.0)
                                                 - st.lognorm.logsf(t64, 0.6, scale=6.0))),
            "lognormal(ln 5, 0.5)": (fs.law("lognormal", math.log(5.0), 0.5),
                                     np.exp(st.lognorm.logpdf(t64, 0.5, scale=5.0) - st.lognorm.logsf(t64, 0.5, scale=5.0))),
            "weibull(2, 4)": (lat, 2.0 / 4.0 * (t64 / 4.0)),
            "erlang(3, 0.75)": (fs.law("erlang", 0.75, k=3),
                                np.exp(st.gamma.logpdf(t64, 3, scale=1 / 0.75) - st.gamma.logsf(t64, 3, scale=1 / 0.75)))}
    herr = {}
    for name, (lw, ref) in refs.items():
        td = torch.from_numpy(tau).cuda()
        hd = torch.empty_like(td)
        fs.fs_eval_hazard(lw, td, hd)
        torch.cuda.synchronize()
        h = hd.cpu().numpy().astype(np.float64)
        ok = ref >= 1e-30
        herr[name] = float(np.max(np.abs(h[ok] - ref[ok]) / ref[ok]))
    out["hazard_max_rel_err"] = {k: float(f"{v:.3g}") for k, v in herr.items()}
    return out


def run_reference(args, rank, world):
    """The oracle timed on every host core on bounded samples of the workload
    (one independent realisation per core; each benchmark step advances every
    realisation by the same number of oracle steps)."""
    if rank != 0:
        return None
    g, idx, wname = workload("regular", args.n)
    h = HostOracle(g, idx)
    per_step = 10   # oracle steps per realisation per benchmark step (a bounded sample)
    times, upd, k = [], 0, 0
    try:
        for it in range(args.warmup + args.steps):
            u, wall, _ = h.advance(per_step)
            k += per_step
            if it >= args.warmup:
                times.append(wall)
                upd += u
    finally:
        h.close()
    total = float(np.sum(times))
    value = upd / total / 1e9
    sample = (f"{h.workers} processes, one per host core, each the single-threaded C oracle on its own "
              f"realisation; {per_step} consecutive oracle steps per realisation per benchmark step, steps "
              f"{args.warmup * per_step} to {k - 1} of the {g.n}-node run")
    return {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wname, "model": "SEIR renewal", "n": g.n, "sim_steps": args.sim_steps,
                       "parallelism": f"host x{h.workers}", "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": h.workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def shedding_bench(fs, torch, n: int, sim_steps: int, graph_steps: int, reps: int = 3):
    """Cost of the age-dependent source infectivity (Eq. 8) on the step, as the
    paper's shedding-overhead table measures it: N = 10^6, mean degree 8, a
    regular and a Barabasi-Albert (m = 4) graph, the same SEIR model with
    constant beta and with beta s(tau), s = the infectious hazard h_IR (and,
    as a second profile, a log-normal shedding density). A profile changes
    the epidemic and so the work (S node-steps and S-row edges gathered are
    reported beside each time); shed_constant_exact isolates the cost of the
    machinery on the constant-beta trajectory. Each variant: event-
    timed CUDA Graph replays of a full run (ingest and init untimed), median
    of `reps`, L2 flushed before each run."""
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    inf, lat = fs.law("lognormal", math.log(6.0), 0.6), fs.law("weibull", 2.0, 4.0)
    K = graph_steps
    full = sim_steps // K
    variants = [
        ("constant_gather", dict(pressure=fs.FS_PRESSURE_GATHER)),
        ("constant_push", dict(pressure=fs.FS_PRESSURE_PUSH)),
        # s = the hazard of Exp(2) = 2 with beta / 2: rho = beta exactly, so the
        # trajectory (and the work) is constant_gather's, bit for bit; the
        # difference is the cost of the infectivity machinery alone
        ("shed_constant_exact", dict(shed_mode=fs.FS_SHED_HAZARD, shedding=fs.law("exp", 2.0))),
        ("shed_hazard_IR", dict(shed_mode=fs.FS_SHED_HAZARD, shedding=inf)),
        ("shed_density_lognormal", dict(shed_mode=fs.FS_SHED_DENSITY, shedding=fs.law("lognormal", math.log(5.0), 0.5))),
    ]
    graphs = [("regular-d8", W.random_regular(n, 8, seed=0)), ("ba-m4", W.barabasi_albert(n, 4, seed=0))]
    res = {"workload": f"seir-shedding-overhead-n{n:.0e}".replace("+0", ""), "sim_steps": sim_steps,
           "graph_steps": K, "timed": "CUDA Graph replays of the step loop (CUDA events), median of runs",
           "graphs": {}}
    for gname, g in graphs:
        allowed = W.non_hub_nodes(g) if gname.startswith("ba") else None
        idx = W.index_nodes(g.n, 100, seed=1, allowed=allowed)
        gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
        row = {}
        for label, kw in variants:
            beta = 0.125 if label == "shed_constant_exact" else 0.25
            prm = fs.sim_params(fs.FS_SEIR, inf, beta, 0.1, 3, latent=lat, **kw)
            times = []
            for r in range(reps + 1):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                sh = fs.fs_sim_init(gh, prm, idx)
                ms = fs.fs_sim_run_timed(sh, sim_steps, K, None)
                c = fs.fs_sim_run(sh, 0)
                work = fs.fs_sim_work(sh)
                fs.fs_sim_destroy(sh)
                if r:
                    times.append(float(np.sum(ms[:full])))
            t = float(np.median(times))
            row[label] = {"value": round(g.n * full * K / (t * 1e-3) / 1e9, 3), "unit": UNIT,
                          "ms_per_run": round(t, 3), "final_R": int(c[-1, 3]),
                          "s_node_steps": int(work["s_node_sum"]), "s_row_edges": int(work["s_degree_sum"])}
        base = row["constant_gather"]["value"]
        for label in ("shed_constant_exact", "shed_hazard_IR", "shed_density_lognormal"):
            row[label]["slowdown_vs_constant_gather_pct"] = round((base / row[label]["value"] - 1) * 100, 2)
        # the s = h_IR profile in a packed ensemble of 8 replicates against the
        # same 8 realisations run alone (host wall clock around the synchronous
        # run calls; ensemble and sims created outside the timed region)
        prms = [fs.sim_params(fs.FS_SEIR, inf, 0.25, 0.1, 3, latent=lat, replicate=r,
                              pressure=fs.FS_PRESSURE_GATHER, shed_mode=fs.FS_SHED_HAZARD, shedding=inf)
                for r in range(8)]
        t_pack, t_alone = [], []
        for r in range(reps + 1):
            e = fs.fs_ens_create(gh, prms, idx)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fs.fs_ens_run(e, sim_steps, 8, K, want_counts=False)
            t1 = time.perf_counter()
            fs.fs_ens_destroy(e)
            alone = 0.0
            for p_ in prms:
                sh = fs.fs_sim_init(gh, p_, idx)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                fs.fs_sim_run(sh, sim_steps, graph_steps=K)
                alone += time.perf_counter() - t2
                fs.fs_sim_destroy(sh)
            if r:
                t_pack.append(t1 - t0)
                t_alone.append(alone)
        tp, ta = float(np.median(t_pack)), float(np.median(t_alone))
        row["packed_shed_hazard_IR_x8"] = {
            "value": round(8 * g.n * sim_steps / tp / 1e9, 3), "unit": UNIT, "seconds": round(tp, 4),
            "alone_value": round(8 * g.n * sim_steps / ta / 1e9, 3), "alone_seconds": round(ta, 4),
            "speedup": round(ta / tp, 2),
            "timed": "8 replicates packed (fs_ens_run) vs each run alone (fs_sim_run), host wall clock"}
        res["graphs"][gname] = row
        fs.fs_graph_destroy(gh)
    return res


def compaction_bench(fs, torch, n: int, sim_steps: int, graph_steps: int, reps: int = 3):
    """Active-node compaction (Section 5.6) as the paper's compaction table
    measures it: N = 10^6, Erdos-Renyi mean degree 8 and Barabasi-Albert m = 4,
    the same SEIR model, TF = sim_steps * dt, each run with and without
    FS_ACTIVE_LIST in the gather form with every node in the one-lane-per-node
    class (the paper's forced configuration), the gather form with the
    automatic class split, and the push form. Event-timed CUDA Graph replays
    (the per-window refreshes included), median of `reps`, L2 flushed."""
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    inf, lat = fs.law("lognormal", math.log(6.0), 0.6), fs.law("weibull", 2.0, 4.0)
    K = graph_steps
    full = sim_steps // K
    res = {"workload": f"seir-compaction-n{n:.0e}".replace("+0", ""), "sim_steps": sim_steps, "graph_steps": K,
           "timed": "CUDA Graph replays incl. refreshes (CUDA events), median of runs", "graphs": {}}
    for gname, g in (("er-d8", W.erdos_renyi(n, 8, seed=0)), ("ba-m4", W.barabasi_albert(n, 4, seed=0))):
        idx = W.index_nodes(g.n, 100, seed=1, allowed=W.non_hub_nodes(g) if gname.startswith("ba") else None)
        row = {}
        for cname, dispatch, pressure in (("gather_thread", fs.FS_DISPATCH_THREAD, fs.FS_PRESSURE_GATHER),
                                          ("gather_auto", fs.FS_DISPATCH_AUTO, fs.FS_PRESSURE_GATHER),
                                          ("push_auto", fs.FS_DISPATCH_AUTO, fs.FS_PRESSURE_PUSH)):
            gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(dispatch, 0))
            cell = {}
            for label, flag in (("baseline", 0), ("compaction", fs.FS_ACTIVE_LIST)):
                prm = fs.sim_params(fs.FS_SEIR, inf, 0.25, 0.1, 3, latent=lat, pressure=pressure | flag)
                times = []
                for r in range(reps + 1):
                    flush.fill_(1.0)
                    torch.cuda.synchronize()
                    sh = fs.fs_sim_init(gh, prm, idx)
                    ms = fs.fs_sim_run_timed(sh, sim_steps, K, None)
                    c = fs.fs_sim_run(sh, 0)
                    listed, units = fs.fs_sim_active_units(sh)
                    fs.fs_sim_destroy(sh)
                    if r:
                        times.append(float(np.sum(ms[:full])))
                t = float(np.median(times))
                cell[label] = {"value": round(g.n * full * K / (t * 1e-3) / 1e9, 3), "unit": UNIT,
                               "ms_per_run": round(t, 3), "final_R_frac": round(int(c[-1, 3]) / g.n, 4)}
                if units:
                    cell[label]["mean_units_visited_frac"] = round(listed / (units * (full + (sim_steps % K > 0))), 4)
            cell["speedup"] = round(cell["compaction"]["value"] / cell["baseline"]["value"], 3)
            row[cname] = cell
            fs.fs_graph_destroy(gh)
        res["graphs"][gname] = row
    return res


def markov_bench(fs, torch, n: int, sim_steps: int, graph_steps: int, reps: int = 3):
    """The Markovian engine (Section 4, Algorithm 1) on the paper's
    Markovian workload shape: Erdos-Renyi mean degree 8, beta = 0.25,
    recovery 0.15, theta = 0.01, p_max = 0.1, tau_max = 0.1, 10 seeds per
    10^3 nodes; SIS and SIR; `sim_steps` steps from the initial state
    (event-timed CUDA Graph replays, ingest and init untimed, median of
    `reps`). Transitions per second is the paper's Markovian figure
    (1.95 * 10^7 / s at N = 10^6 on its hardware)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    g = W.erdos_renyi(n, 8, seed=0)
    idx = W.index_nodes(g.n, max(1, n // 100), seed=1)
    K = graph_steps
    full = sim_steps // K
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    res = {"workload": f"markov-er8-n{n:.0e}".replace("+0", ""), "sim_steps": full * K, "graph_steps": K,
           "theta": 0.01, "p_max": 0.1, "tau_max": 0.1,
           "timed": "CUDA Graph replays (3 launches per step), median of runs", "models": {}}
    for mname, model in (("sis", fs.FS_SIS), ("sir", fs.FS_SIR)):
        prm = fs.sim_params(model, fs.law("exp", 0.15), 0.25, 0.1, 3, theta=0.01, p_max=0.1)
        rows = []
        for r in range(reps + 1):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            sh = fs.fs_sim_init(gh, prm, idx)
            ms = fs.fs_sim_run_timed(sh, full * K, K, None)
            trans = fs.fs_sim_transitions(sh)
            t_sim = fs.fs_sim_time(sh)[0]
            c = fs.fs_sim_run(sh, 0)
            fs.fs_sim_destroy(sh)
            if r:
                rows.append((float(np.sum(ms[:full])), trans, t_sim, c[-1]))
        rows.sort(key=lambda x: x[0])
        t_ms, trans, t_sim, cnt = rows[len(rows) // 2]
        res["models"][mname] = {
            "transitions_per_s": round(trans / (t_ms * 1e-3), 1), "transitions": int(trans),
            "node_updates_per_s": round(g.n * full * K / (t_ms * 1e-3), 1), "ms_per_run": round(t_ms, 3),
            "us_per_step": round(t_ms * 1e3 / (full * K), 3), "simulated_days": round(t_sim, 3),
            "final_counts": [int(v) for v in cnt]}
    fs.fs_graph_destroy(gh)
    return res


def run_extra(args):
    """Full-size packed-ensemble or serving runs (their own JSON line)."""
    import torch
    import paper_2604_22092_gb300 as fs
    fs.load()
    age = fs.FS_AGE_F16 if args.age == "f16" else fs.FS_AGE_F32
    if args.workload == "ensemble":
        res = ensemble_bench(fs, torch, n_graphs=args.ens_graphs, n_lo=1e4, n_hi=2e6, steps=args.ens_steps,
                             age_dtype=age, pressure=PRESSURE[args.pressure])
    elif args.workload == "precision":
        res = precision_bench(fs, torch, n=args.n, steps=args.sim_steps, reps=1000)
    elif args.workload == "markov":
        res = markov_bench(fs, torch, n=args.n, sim_steps=args.sim_steps, graph_steps=args.graph_steps)
    elif args.workload == "compaction":
        res = compaction_bench(fs, torch, n=args.n, sim_steps=args.sim_steps, graph_steps=args.graph_steps)
    elif args.workload == "shedding":
        res = shedding_bench(fs, torch, n=args.n, sim_steps=args.sim_steps, graph_steps=args.graph_steps)
    elif args.workload == "large":
        sizes = ((10_000_000, fs.FS_AGE_F32), (100_000_000, fs.FS_AGE_F32), (100_000_000, fs.FS_AGE_BF16))
        if args.large_n:
            sizes = tuple((int(float(v)), fs.FS_AGE_F32) for v in args.large_n.split(","))
        for n, a in sizes:
            res = large_bench(fs, torch, n, a, args.sim_steps, args.graph_steps, reps=1,
                              pressure=PRESSURE[args.pressure])
            print(json.dumps({"metric": METRIC, "impl": "flashstep", "data": "synthetic", **res}), flush=True)
        return
    else:
        # C4's shape scaled to a few minutes: request graphs up to N = 10^7,
        # beside the N = 10^8 SEIR job with BF16 ages
        res = serving_bench(fs, torch, n_requests=args.serve_requests, n_pool=16, n_hi=1e7, steps=200, rep_lo=16,
                            rep_hi=256, window_s=args.serve_requests / 40.0, age_dtype=age, big_n=1e8,
                            big_age=fs.FS_AGE_BF16)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "impl": "flashstep", "data": "synthetic", **res}), flush=True)


# ------------------------------------------------------------------ ranks
def rank_setup(environ, gpus: int):
    """(rank, world, local_rank) of this process, and the environment changes
    it needs. Under torchrun every rank is one replica on its own GPU: that GPU
    is made the only visible one, so that every CUDA runtime in the process
    (torch's and the library's) addresses the same device."""
    changes = {}
    world = int(environ.get("WORLD_SIZE", "1"))
    local_rank = int(environ.get("LOCAL_RANK", "0"))
    if world > 1 and "LOCAL_RANK" in environ:
        changes = {"CUDA_VISIBLE_DEVICES": environ["LOCAL_RANK"], "LOCAL_RANK": "0"}
        local_rank = 0
    rank = int(environ.get("RANK", "0"))
    if "WORLD_SIZE" not in environ:
        world = gpus if gpus == 1 else 1
    return rank, world, local_rank, changes


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (a job lasts as long as its slowest
    rank); the value itself when there is one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gnups(n: int, sim_steps: int, bench_steps: int, world: int, total_ms: float) -> float:
    """Node updates of all replicas (weak scaling: every rank runs the full
    workload on its own GPU) per second of the slowest rank, in GNUPS."""
    return n * sim_steps * bench_steps * world / (total_ms * 1e-3) / 1e9


def replica_seed(rank: int) -> int:
    """Philox seed of rank r's replica: distinct realisations, no exchange."""
    return 1 + rank


def main():
    args = parse()
    if args.workload != "regular":
        run_extra(args)
        return
    rank, world, local_rank, changes = rank_setup(os.environ, args.gpus)
    os.environ.update(changes)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_flashstep(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
