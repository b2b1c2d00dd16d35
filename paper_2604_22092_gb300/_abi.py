"""ctypes mirror of include/fs.h (structures, enums and prototypes).

Argument marshalling only: every computation happens in libflashstep.so.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import _build_lib

FS_OK, FS_EINVAL, FS_ENOMEM, FS_ECUDA, FS_ETIMEOUT, FS_EBUSY, FS_ESTATE, FS_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "FS_OK", 1: "FS_EINVAL", 2: "FS_ENOMEM", 3: "FS_ECUDA", 4: "FS_ETIMEOUT",
                5: "FS_EBUSY", 6: "FS_ESTATE", 7: "FS_EUNSUPPORTED"}
FS_S, FS_E, FS_I, FS_R = 0, 1, 2, 3
FS_SIR, FS_SEIR, FS_SIS = 0, 1, 2
FS_AGE_F32, FS_AGE_F16, FS_AGE_BF16 = 0, 1, 2
FS_DISPATCH_AUTO, FS_DISPATCH_THREAD, FS_DISPATCH_MERGE, FS_DISPATCH_TUNE = 0, 1, 2, 3
FS_PRESSURE_AUTO, FS_PRESSURE_GATHER, FS_PRESSURE_PUSH = 0, 1, 2
FS_SHED_NONE, FS_SHED_HAZARD, FS_SHED_DENSITY = 0, 1, 2
FS_ACTIVE_LIST = 0x4
FS_LAW_NONE, FS_LAW_EXP, FS_LAW_LOGNORMAL, FS_LAW_WEIBULL, FS_LAW_ERLANG = 0, 1, 2, 3, 4
FS_TEST_WAIT_TIMEOUT, FS_TEST_BOUNDS_SHRINK = 1, 2


class fs_law(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double)]


class fs_sim_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("age_dtype", ctypes.c_int32),
                ("latent", fs_law), ("infectious", fs_law),
                ("beta", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("replicate", ctypes.c_uint32),
                ("index_state", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("shed_mode", ctypes.c_int32), ("eps", ctypes.c_double), ("delta", ctypes.c_double),
                ("shedding", fs_law), ("theta", ctypes.c_double), ("p_max", ctypes.c_double),
                ("markov_mode", ctypes.c_int32), ("reserved2_", ctypes.c_int32)]


class fs_graph_opts(ctypes.Structure):
    _fields_ = [("dispatch", ctypes.c_int32), ("thread_max_deg", ctypes.c_int32),
                ("device_input", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class fs_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("d_max", ctypes.c_int64),
                ("d_avg", ctypes.c_double), ("rho", ctypes.c_double),
                ("n_thread", ctypes.c_int64), ("n_merge", ctypes.c_int64),
                ("sell_entries", ctypes.c_int64), ("merge_chunks", ctypes.c_int64),
                ("thread_max_deg", ctypes.c_int32), ("identity_layout", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class fs_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_members", ctypes.c_int32),
                ("quantum", ctypes.c_int32), ("age_dtype", ctypes.c_int32), ("reserved_", ctypes.c_int32),
                ("max_inflight", ctypes.c_int64), ("wait_limit_s", ctypes.c_double)]


class fs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("running", ctypes.c_int64), ("launches", ctypes.c_int64), ("node_updates", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("busy_seconds", ctypes.c_double)]


VP = ctypes.c_void_p
P = ctypes.POINTER
# fs_alloc_fn / fs_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# name -> (restype, argtypes); the exported C ABI
PROTOTYPES = {
    "fs_version": (ctypes.c_char_p, []),
    "fs_last_error": (ctypes.c_char_p, []),
    "fs_graph_create": (ctypes.c_int, [ctypes.c_int64, VP, VP, VP, P(fs_graph_opts), VP, P(VP)]),
    "fs_graph_info": (ctypes.c_int, [VP, P(fs_graph_info)]),
    "fs_graph_info_get": (ctypes.c_int, [VP, P(fs_graph_info)]),
    "fs_graph_destroy": (ctypes.c_int, [VP]),
    "fs_test_inject": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "fs_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, VP]),
    "fs_ens_time": (ctypes.c_int, [VP, VP, VP]),
    "fs_release_cached_memory": (ctypes.c_int, []),
    "fs_cached_memory": (ctypes.c_int, [P(ctypes.c_uint64), P(ctypes.c_uint64)]),
    "fs_debug_bounds_build": (ctypes.c_int, [P(ctypes.c_int32)]),
    "fs_sim_init": (ctypes.c_int, [VP, P(fs_sim_params), VP, ctypes.c_int64, VP, P(VP)]),
    "fs_sim_step": (ctypes.c_int, [VP, VP]),
    "fs_sim_run": (ctypes.c_int, [VP, ctypes.c_int64, ctypes.c_int32, VP]),
    "fs_sim_run_async": (ctypes.c_int, [VP, ctypes.c_int64, ctypes.c_int32, VP]),
    "fs_sim_sync": (ctypes.c_int, [VP]),
    "fs_sim_run_timed": (ctypes.c_int, [VP, ctypes.c_int64, ctypes.c_int32, VP, VP, P(ctypes.c_int64)]),
    "fs_kernel_launches": (ctypes.c_int, [P(ctypes.c_uint64)]),
    "fs_sim_get_state": (ctypes.c_int, [VP, VP, VP, P(ctypes.c_int64)]),
    "fs_sim_set_state": (ctypes.c_int, [VP, VP, VP, ctypes.c_int64]),
    "fs_sim_work": (ctypes.c_int, [VP, P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_int64)]),
    "fs_sim_pressure_get": (ctypes.c_int, [VP, P(ctypes.c_int32)]),
    "fs_ens_pressure_get": (ctypes.c_int, [VP, P(ctypes.c_int32)]),
    "fs_sim_time": (ctypes.c_int, [VP, P(ctypes.c_double), P(ctypes.c_float)]),
    "fs_sim_infectivity_get": (ctypes.c_int, [VP, VP]),
    "fs_sim_active_units": (ctypes.c_int, [VP, P(ctypes.c_uint64), P(ctypes.c_uint64)]),
    "fs_sim_transitions": (ctypes.c_int, [VP, P(ctypes.c_uint64)]),
    "fs_sim_destroy": (ctypes.c_int, [VP]),
    "fs_eval_hazard": (ctypes.c_int, [P(fs_law), VP, VP, ctypes.c_int64, VP]),
    "fs_eval_density": (ctypes.c_int, [P(fs_law), VP, VP, ctypes.c_int64, VP]),
    "fs_eval_uniforms": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, VP, VP,
                                        ctypes.c_int64, VP]),
    "fs_step_noalloc": (ctypes.c_int, [VP, P(fs_sim_params), ctypes.c_int64, VP, VP, VP, VP, VP, VP]),
    "fs_ens_create": (ctypes.c_int, [VP, P(fs_sim_params), ctypes.c_int32, VP, ctypes.c_int64, P(VP)]),
    "fs_ens_run": (ctypes.c_int, [VP, ctypes.c_int64, ctypes.c_int32, VP]),
    "fs_ens_get_state": (ctypes.c_int, [VP, ctypes.c_int32, VP, VP, P(ctypes.c_int64)]),
    "fs_ens_destroy": (ctypes.c_int, [VP]),
    "fs_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, VP, P(VP)]),
    "fs_batch_add": (ctypes.c_int, [VP, VP, ctypes.c_int64, VP]),
    "fs_batch_run": (ctypes.c_int, [VP, ctypes.c_int64, ctypes.c_int32]),
    "fs_batch_status": (ctypes.c_int, [VP, P(ctypes.c_int32), P(ctypes.c_int64)]),
    "fs_batch_destroy": (ctypes.c_int, [VP]),
    "fs_tune_stats": (ctypes.c_int, [P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)]),
    "fs_tune_reset": (ctypes.c_int, []),
    "fs_server_create": (ctypes.c_int, [P(fs_server_cfg), P(VP)]),
    "fs_server_submit": (ctypes.c_int, [VP, VP, P(fs_sim_params), ctypes.c_int32, ctypes.c_int32, VP,
                                        ctypes.c_int64, ctypes.c_int64, P(ctypes.c_uint64)]),
    "fs_server_poll": (ctypes.c_int, [VP, ctypes.c_uint64, P(ctypes.c_int32), VP, P(ctypes.c_double)]),
    "fs_server_drain": (ctypes.c_int, [VP, ctypes.c_double]),
    "fs_server_stats_get": (ctypes.c_int, [VP, P(fs_server_stats)]),
    "fs_server_destroy": (ctypes.c_int, [VP]),
}

_lib = None


def lib_path() -> str:
    return _build_lib.LIB


def load(build_if_missing: bool = True):
    """Load libflashstep.so (building it first if asked and stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build_lib.is_fresh():
        _build_lib.build()
    path = _build_lib.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libflashstep.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class FsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def check(status: int, where: str) -> None:
    if status != FS_OK:
        msg = load().fs_last_error().decode(errors="replace")
        raise FsError(status, where, msg)
