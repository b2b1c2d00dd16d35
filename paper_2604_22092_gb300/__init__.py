"""flashstep: the renewal (age-dependent hazard) Bernoulli tau-leaping step of
SIR/SEIR on a CSR contact graph, as hand-written CUDA for GB300 (sm_103a),
after FlashSpread (arXiv 2604.22092).

This module is a thin binding of the C ABI in include/fs.h: every function
has the name of the C entry point it calls and only marshals arguments
(numpy arrays for host buffers, torch CUDA tensors or raw integers for device
buffers and streams). All computation runs in libflashstep.so; if the library
is missing the import of any entry point raises.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _abi
from ._abi import (FS_AGE_BF16, FS_AGE_F16, FS_AGE_F32, FS_DISPATCH_AUTO, FS_DISPATCH_MERGE,
                   FS_DISPATCH_THREAD, FS_DISPATCH_TUNE, FS_E, FS_I, FS_LAW_ERLANG, FS_LAW_EXP, FS_LAW_LOGNORMAL,
                   FS_LAW_NONE, FS_LAW_WEIBULL, FS_PRESSURE_AUTO, FS_PRESSURE_GATHER, FS_PRESSURE_PUSH, FS_R,
                   FS_S, FS_SEIR, FS_SHED_DENSITY, FS_SHED_HAZARD, FS_SHED_NONE, FS_SIR, FS_SIS, FS_ACTIVE_LIST,
                   FS_TEST_BOUNDS_SHRINK, FS_TEST_WAIT_TIMEOUT, FsError, check)

__all__ = [
    "fs_version", "fs_last_error", "fs_graph_create", "fs_graph_info", "fs_graph_info_get", "fs_graph_destroy",
    "fs_sim_init", "fs_sim_step", "fs_sim_run", "fs_sim_run_async", "fs_sim_sync", "fs_sim_run_timed",
    "fs_kernel_launches", "fs_tune_stats", "fs_tune_reset",
    "fs_sim_get_state", "fs_sim_set_state", "fs_sim_work", "fs_sim_pressure_get", "fs_ens_pressure_get", "fs_sim_time",
    "fs_sim_infectivity_get", "fs_sim_active_units", "fs_sim_transitions", "fs_sim_destroy",
    "fs_eval_hazard", "fs_eval_density",
    "fs_eval_uniforms", "fs_step_noalloc", "fs_ens_create", "fs_ens_run", "fs_ens_get_state", "fs_ens_time",
    "fs_ens_destroy", "fs_batch_create", "fs_batch_add", "fs_batch_run", "fs_batch_status", "fs_batch_destroy",
    "fs_server_create", "fs_server_submit", "fs_server_poll", "fs_server_drain", "fs_server_stats_get",
    "fs_server_destroy", "fs_test_inject", "fs_debug_bounds_build", "fs_set_allocator",
    "fs_release_cached_memory", "fs_cached_memory",
    "law", "sim_params", "graph_opts", "FsError", "load",
    "FS_S", "FS_E", "FS_I", "FS_R", "FS_SIR", "FS_SEIR", "FS_SIS", "FS_AGE_F32", "FS_AGE_F16", "FS_AGE_BF16",
    "FS_DISPATCH_AUTO", "FS_DISPATCH_THREAD", "FS_DISPATCH_MERGE", "FS_DISPATCH_TUNE",
    "FS_PRESSURE_AUTO", "FS_PRESSURE_GATHER", "FS_PRESSURE_PUSH", "FS_SHED_NONE", "FS_SHED_HAZARD",
    "FS_SHED_DENSITY", "FS_ACTIVE_LIST", "FS_TEST_WAIT_TIMEOUT", "FS_TEST_BOUNDS_SHRINK",
]


def load():
    """Load (building if stale) libflashstep.so; returns the ctypes library."""
    return _abi.load()


def _addr(x):
    """Address of a buffer: numpy array (host), torch tensor (device/host), int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s or None
    return s.cuda_stream or None


# --------------------------------------------------------------- parameters
def law(kind: str, a: float = 0.0, b: float = 0.0, k: int = 0) -> _abi.fs_law:
    """Holding-time law: exp(rate), lognormal(mu, sigma), weibull(shape, scale),
    erlang(rate, k=stages), none."""
    code = {"none": FS_LAW_NONE, "exp": FS_LAW_EXP, "lognormal": FS_LAW_LOGNORMAL,
            "weibull": FS_LAW_WEIBULL, "erlang": FS_LAW_ERLANG}[kind]
    return _abi.fs_law(code, int(k), float(a), float(b))


def sim_params(model: int, infectious: _abi.fs_law, beta: float, dt: float, seed: int,
               latent: _abi.fs_law | None = None, replicate: int = 0, index_state: int | None = None,
               age_dtype: int = FS_AGE_F32, pressure: int = FS_PRESSURE_AUTO, eps: float = 0.0,
               delta: float = 0.0, shed_mode: int = FS_SHED_NONE,
               shedding: _abi.fs_law | None = None, theta: float = 0.0, p_max: float = 0.0,
               markov_mode: int = 0) -> _abi.fs_sim_params:
    """pressure: FS_PRESSURE_AUTO / FS_PRESSURE_GATHER / FS_PRESSURE_PUSH, optionally
    | FS_ACTIVE_LIST (the flags field);
    eps > 0: adaptive step with dt as its cap (delta 0 = 1e-12);
    shed_mode / shedding: the shedding profile s(tau) of the infectivity (FS_SHED_NONE: s = 1);
    theta > 0: the Markovian engine (Algorithm 1) with p_max (0 = 0.1) and dt as tau_max."""
    if index_state is None:
        index_state = FS_E if model == FS_SEIR else FS_I
    return _abi.fs_sim_params(int(model), int(age_dtype), latent if latent is not None else law("none"),
                              infectious, float(beta), float(dt), int(seed), int(replicate),
                              int(index_state), int(pressure), int(shed_mode), float(eps), float(delta),
                              shedding if shedding is not None else law("none"), float(theta), float(p_max),
                              int(markov_mode), 0)


def graph_opts(dispatch: int = FS_DISPATCH_AUTO, thread_max_deg: int = 0,
               device_input: bool = False) -> _abi.fs_graph_opts:
    return _abi.fs_graph_opts(int(dispatch), int(thread_max_deg), 1 if device_input else 0, 0)


# --------------------------------------------------------------- entry points
def fs_version() -> str:
    return load().fs_version().decode()


def fs_last_error() -> str:
    return load().fs_last_error().decode(errors="replace")


def fs_graph_create(n: int, row_ptr, col_ind, weights=None, opts: _abi.fs_graph_opts | None = None,
                    stream=None) -> int:
    """Returns an opaque graph handle. row_ptr/col_ind: numpy int64/int32 on the
    host, or torch CUDA tensors with opts.device_input = 1."""
    L = load()
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_ind = np.ascontiguousarray(col_ind, dtype=np.int32)
    h = ctypes.c_void_p()
    st = L.fs_graph_create(int(n), _addr(row_ptr), _addr(col_ind), _addr(weights),
                           ctypes.byref(opts) if opts is not None else None, _stream(stream),
                           ctypes.byref(h))
    check(st, "fs_graph_create")
    return h.value


def fs_graph_info(g: int) -> dict:
    info = _abi.fs_graph_info()
    check(load().fs_graph_info(g, ctypes.byref(info)), "fs_graph_info")
    return {name: getattr(info, name) for name, _ in info._fields_}


def fs_graph_info_get(g: int) -> dict:
    info = _abi.fs_graph_info()
    check(load().fs_graph_info_get(g, ctypes.byref(info)), "fs_graph_info_get")
    return {name: getattr(info, name) for name, _ in info._fields_}


def fs_graph_destroy(g: int) -> None:
    check(load().fs_graph_destroy(g), "fs_graph_destroy")


def fs_sim_init(g: int, params: _abi.fs_sim_params, index_nodes, stream=None) -> int:
    idx = np.ascontiguousarray(index_nodes, dtype=np.int32)
    h = ctypes.c_void_p()
    st = load().fs_sim_init(g, ctypes.byref(params), _addr(idx) if idx.size else None, idx.size,
                            _stream(stream), ctypes.byref(h))
    check(st, "fs_sim_init")
    return h.value


def fs_sim_step(s: int) -> np.ndarray:
    c = np.zeros(4, dtype=np.uint32)
    check(load().fs_sim_step(s, _addr(c)), "fs_sim_step")
    return c


def fs_sim_run(s: int, steps: int, graph_steps: int = 0, want_counts: bool = True):
    c = np.zeros((steps + 1, 4), dtype=np.uint32) if want_counts else None
    check(load().fs_sim_run(s, int(steps), int(graph_steps), _addr(c)), "fs_sim_run")
    return c


def fs_sim_run_async(s: int, steps: int, graph_steps: int = 0, counts_dev=None) -> None:
    check(load().fs_sim_run_async(s, int(steps), int(graph_steps), _addr(counts_dev)), "fs_sim_run_async")


def fs_sim_sync(s: int) -> None:
    check(load().fs_sim_sync(s), "fs_sim_sync")


def fs_sim_run_timed(s: int, steps: int, graph_steps: int = 0, counts_dev=None) -> np.ndarray:
    """Runs `steps` steps and returns the event-timed ms of every graph replay
    (and, last, of the directly launched remainder)."""
    K = graph_steps or 50
    ms = np.zeros(steps // K + 1, dtype=np.float32)
    n = ctypes.c_int64()
    check(load().fs_sim_run_timed(s, int(steps), int(graph_steps), _addr(counts_dev), _addr(ms),
                                  ctypes.byref(n)), "fs_sim_run_timed")
    return ms[:n.value]


def fs_tune_stats() -> dict:
    t, h, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(load().fs_tune_stats(ctypes.byref(t), ctypes.byref(h), ctypes.byref(p)), "fs_tune_stats")
    return {"trials": t.value, "cache_hits": h.value, "profiles": p.value}


def fs_tune_reset() -> None:
    check(load().fs_tune_reset(), "fs_tune_reset")


def fs_kernel_launches() -> int:
    c = ctypes.c_uint64()
    check(load().fs_kernel_launches(ctypes.byref(c)), "fs_kernel_launches")
    return c.value


_AGE_NP = {FS_AGE_F32: np.float32, FS_AGE_F16: np.uint16, FS_AGE_BF16: np.uint16}


def fs_sim_get_state(s: int, n: int, age_dtype: int = FS_AGE_F32):
    """(state uint8[n], age[n] (float32, or the raw 16-bit storage), step)."""
    X = np.zeros(n, dtype=np.uint8)
    A = np.zeros(n, dtype=_AGE_NP[age_dtype])
    step = ctypes.c_int64()
    check(load().fs_sim_get_state(s, _addr(X), _addr(A), ctypes.byref(step)), "fs_sim_get_state")
    return X, A, step.value


def fs_sim_set_state(s: int, state, age, step: int) -> None:
    X = np.ascontiguousarray(state, dtype=np.uint8)
    A = np.ascontiguousarray(age)
    check(load().fs_sim_set_state(s, _addr(X), _addr(A), int(step)), "fs_sim_set_state")


def fs_sim_work(s: int) -> dict:
    ds, sn, k = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int64()
    check(load().fs_sim_work(s, ctypes.byref(ds), ctypes.byref(sn), ctypes.byref(k)), "fs_sim_work")
    return {"s_degree_sum": ds.value, "s_node_sum": sn.value, "steps": k.value}


def fs_sim_time(s: int) -> tuple[float, float]:
    """(elapsed simulated time, size of the next step)."""
    t, d = ctypes.c_double(), ctypes.c_float()
    check(load().fs_sim_time(s, ctypes.byref(t), ctypes.byref(d)), "fs_sim_time")
    return t.value, d.value


def fs_sim_infectivity_get(s: int, n: int, age_dtype: int = FS_AGE_F32) -> np.ndarray:
    """rho[n] the next step reads (float32, or the raw 16-bit storage); 0 for non-I nodes."""
    rho = np.zeros(n, dtype=_AGE_NP[age_dtype])
    check(load().fs_sim_infectivity_get(s, _addr(rho)), "fs_sim_infectivity_get")
    return rho


def fs_sim_active_units(s: int) -> tuple[int, int]:
    """(units visited summed over launch sequences, units per sequence) of FS_ACTIVE_LIST."""
    a, u = ctypes.c_uint64(), ctypes.c_uint64()
    check(load().fs_sim_active_units(s, ctypes.byref(a), ctypes.byref(u)), "fs_sim_active_units")
    return a.value, u.value


def fs_sim_transitions(s: int) -> int:
    """Node transitions of the steps run since init or set_state."""
    t = ctypes.c_uint64()
    check(load().fs_sim_transitions(s, ctypes.byref(t)), "fs_sim_transitions")
    return t.value


def fs_ens_pressure_get(e: int) -> int:
    """FS_PRESSURE_GATHER or FS_PRESSURE_PUSH: the form the ensemble runs."""
    v = ctypes.c_int32()
    check(load().fs_ens_pressure_get(e, ctypes.byref(v)), "fs_ens_pressure_get")
    return v.value


def fs_sim_pressure_get(s: int) -> int:
    """FS_PRESSURE_GATHER or FS_PRESSURE_PUSH: the form the sim runs."""
    v = ctypes.c_int32()
    check(load().fs_sim_pressure_get(s, ctypes.byref(v)), "fs_sim_pressure_get")
    return v.value


def fs_sim_destroy(s: int) -> None:
    check(load().fs_sim_destroy(s), "fs_sim_destroy")


def fs_eval_hazard(lw: _abi.fs_law, tau_dev, h_dev, stream=None) -> None:
    n = tau_dev.numel()
    check(load().fs_eval_hazard(ctypes.byref(lw), _addr(tau_dev), _addr(h_dev), n, _stream(stream)),
          "fs_eval_hazard")


def fs_eval_density(lw: _abi.fs_law, tau_dev, f_dev, stream=None) -> None:
    n = tau_dev.numel()
    check(load().fs_eval_density(ctypes.byref(lw), _addr(tau_dev), _addr(f_dev), n, _stream(stream)),
          "fs_eval_density")


def fs_eval_uniforms(seed: int, replicate: int, step: int, nodes_dev, u_dev, stream=None) -> None:
    n = nodes_dev.numel()
    check(load().fs_eval_uniforms(int(seed), int(replicate), int(step), _addr(nodes_dev), _addr(u_dev), n,
                                  _stream(stream)), "fs_eval_uniforms")


def fs_step_noalloc(g: int, params: _abi.fs_sim_params, step: int, state_dev, age_dev, bitmap_cur_dev,
                    bitmap_next_dev, deltas_dev, stream=None) -> None:
    """One step on caller-owned device buffers that allocates no device
    memory (for callers that may not call cudaMalloc, e.g. under stream
    capture or inside their own memory pool). Enqueues only; see fs.h."""
    check(load().fs_step_noalloc(g, ctypes.byref(params), int(step), _addr(state_dev), _addr(age_dev),
                                 _addr(bitmap_cur_dev), _addr(bitmap_next_dev), _addr(deltas_dev),
                                 _stream(stream)), "fs_step_noalloc")


_ALLOCATOR = None    # the C function pointers of the installed allocator, kept alive


def fs_set_allocator(alloc=None, free=None) -> None:
    """Route the library's device allocations to alloc(bytes) -> address (0
    when out of memory) and free(address); None, None restores the library's
    own caching allocator."""
    global _ALLOCATOR
    if (alloc is None) != (free is None):
        raise ValueError("give both functions or neither")
    if alloc is None:
        fa, ff = _abi.ALLOC_FN(), _abi.FREE_FN()
    else:
        fa = _abi.ALLOC_FN(lambda nbytes, ctx: int(alloc(int(nbytes)) or 0))
        ff = _abi.FREE_FN(lambda ptr, ctx: free(int(ptr)))
    check(load().fs_set_allocator(fa, ff, None), "fs_set_allocator")
    _ALLOCATOR = (fa, ff) if alloc is not None else None


def fs_release_cached_memory() -> None:
    check(load().fs_release_cached_memory(), "fs_release_cached_memory")


def fs_cached_memory() -> dict:
    c, b = ctypes.c_uint64(), ctypes.c_uint64()
    check(load().fs_cached_memory(ctypes.byref(c), ctypes.byref(b)), "fs_cached_memory")
    return {"cached_bytes": c.value, "live_blocks": b.value}


def fs_test_inject(what: int, value: int) -> None:
    """Failure-detection test settings for sims created afterwards (fs.h)."""
    check(load().fs_test_inject(int(what), int(value)), "fs_test_inject")


def fs_debug_bounds_build() -> bool:
    e = ctypes.c_int32()
    check(load().fs_debug_bounds_build(ctypes.byref(e)), "fs_debug_bounds_build")
    return bool(e.value)


# --------------------------------------------------------------- ensembles
def fs_ens_time(e: int, n_real: int) -> tuple[np.ndarray, np.ndarray]:
    """(simulated time covered, size of the next step) of every realisation."""
    t = np.zeros(n_real, dtype=np.float64)
    d = np.zeros(n_real, dtype=np.float32)
    check(load().fs_ens_time(e, _addr(t), _addr(d)), "fs_ens_time")
    return t, d


def fs_ens_create(g: int, params, index_nodes) -> int:
    """params: a sequence of fs_sim_params (1..32 realisations of graph g)."""
    arr = (_abi.fs_sim_params * len(params))(*params)
    idx = np.ascontiguousarray(index_nodes, dtype=np.int32)
    h = ctypes.c_void_p()
    check(load().fs_ens_create(g, arr, len(params), _addr(idx) if idx.size else None, idx.size, ctypes.byref(h)),
          "fs_ens_create")
    return h.value


def fs_ens_run(e: int, steps: int, n_real: int, graph_steps: int = 0, want_counts: bool = True):
    c = np.zeros((steps + 1, n_real, 4), dtype=np.uint32) if want_counts else None
    check(load().fs_ens_run(e, int(steps), int(graph_steps), _addr(c)), "fs_ens_run")
    return c


def fs_ens_get_state(e: int, r: int, n: int, age_dtype: int = FS_AGE_F32):
    X = np.zeros(n, dtype=np.uint8)
    A = np.zeros(n, dtype=_AGE_NP[age_dtype])
    step = ctypes.c_int64()
    check(load().fs_ens_get_state(e, int(r), _addr(X), _addr(A), ctypes.byref(step)), "fs_ens_get_state")
    return X, A, step.value


def fs_ens_destroy(e: int) -> None:
    check(load().fs_ens_destroy(e), "fs_ens_destroy")


def fs_batch_create(age_dtype: int = FS_AGE_F32, max_members: int = 1024, stream=None) -> int:
    h = ctypes.c_void_p()
    check(load().fs_batch_create(int(age_dtype), int(max_members), _stream(stream), ctypes.byref(h)),
          "fs_batch_create")
    return h.value


def fs_batch_add(b: int, e: int, steps: int, counts_out=None) -> None:
    """counts_out: None or a host uint32 array of shape (steps+1, n_real, 4),
    written when the member completes."""
    check(load().fs_batch_add(b, e, int(steps), _addr(counts_out)), "fs_batch_add")


def fs_batch_run(b: int, launches: int, graph_steps: int = 0) -> None:
    check(load().fs_batch_run(b, int(launches), int(graph_steps)), "fs_batch_run")


def fs_batch_status(b: int):
    live, need = ctypes.c_int32(), ctypes.c_int64()
    check(load().fs_batch_status(b, ctypes.byref(live), ctypes.byref(need)), "fs_batch_status")
    return live.value, need.value


def fs_batch_destroy(b: int) -> None:
    check(load().fs_batch_destroy(b), "fs_batch_destroy")


# --------------------------------------------------------------- serving
def fs_server_create(hbm_budget_bytes: int = 0, max_members: int = 0, quantum: int = 0,
                     age_dtype: int = FS_AGE_F32, max_inflight: int = 0, wait_limit_s: float = 0.0) -> int:
    cfg = _abi.fs_server_cfg(int(hbm_budget_bytes), int(max_members), int(quantum), int(age_dtype), 0,
                             int(max_inflight), float(wait_limit_s))
    h = ctypes.c_void_p()
    check(load().fs_server_create(ctypes.byref(cfg), ctypes.byref(h)), "fs_server_create")
    return h.value


def fs_server_submit(srv: int, g: int, scenarios, replicates: int, index_nodes, steps: int) -> int:
    arr = (_abi.fs_sim_params * len(scenarios))(*scenarios)
    idx = np.ascontiguousarray(index_nodes, dtype=np.int32)
    rid = ctypes.c_uint64()
    check(load().fs_server_submit(srv, g, arr, len(scenarios), int(replicates), _addr(idx) if idx.size else None,
                                  idx.size, int(steps), ctypes.byref(rid)), "fs_server_submit")
    return rid.value


def fs_server_poll(srv: int, request_id: int, steps: int = 0, n_real: int = 0):
    """(done, counts[(steps+1), n_real, 4] or None, seconds)."""
    done = ctypes.c_int32()
    sec = ctypes.c_double()
    c = np.zeros((steps + 1, n_real, 4), dtype=np.uint32) if n_real else None
    check(load().fs_server_poll(srv, int(request_id), ctypes.byref(done), _addr(c), ctypes.byref(sec)),
          "fs_server_poll")
    return bool(done.value), (c if done.value else None), sec.value


def fs_server_drain(srv: int, timeout_s: float = 600.0) -> None:
    check(load().fs_server_drain(srv, float(timeout_s)), "fs_server_drain")


def fs_server_stats_get(srv: int) -> dict:
    st = _abi.fs_server_stats()
    check(load().fs_server_stats_get(srv, ctypes.byref(st)), "fs_server_stats_get")
    return {name: getattr(st, name) for name, _ in st._fields_}


def fs_server_destroy(srv: int) -> None:
    check(load().fs_server_destroy(srv), "fs_server_destroy")
