"""CPU oracle for the renewal Bernoulli tau-leaping step (test infrastructure).

This package is TEST INFRASTRUCTURE. Only the test suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it;
the product library never loads, links or calls it, and shares no code with
it. It wraps the plain C implementation in ``fs_oracle.c`` (double-precision
hazards, exact emulation of the age storage rounding, Philox4x32-10 uniforms)
with ctypes and numpy.

Every function follows FlashSpread (arXiv 2604.22092): the state model of
Section 3 (Eqs. 1-3), the stable log-normal hazard of Section 5.1
(Proposition 1), the Bernoulli tau-leap of Section 5.2, the fused step of
Algorithm 3 at a fixed step, and the storage contract of Section 5.7.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

S, E, I, R = 0, 1, 2, 3
SIR, SEIR, SIS = 0, 1, 2
LAW_NONE, LAW_EXP, LAW_LOGNORMAL, LAW_WEIBULL, LAW_ERLANG = 0, 1, 2, 3, 4
AGE_F32, AGE_F16, AGE_BF16 = 0, 1, 2
SHED_NONE, SHED_HAZARD, SHED_DENSITY = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, IEEE semantics, no FMA)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "fs_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Law(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("age_dtype", ctypes.c_int32),
                ("latent", Law), ("infectious", Law),
                ("beta", ctypes.c_double), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("rep", ctypes.c_uint32),
                ("shed_mode", ctypes.c_int32), ("shedding", Law)]


def law(kind: str, a: float = 0.0, b: float = 0.0, k: int = 0) -> Law:
    """kind in {none, exp, lognormal, weibull, erlang}; see fs_oracle.h."""
    code = {"none": LAW_NONE, "exp": LAW_EXP, "lognormal": LAW_LOGNORMAL,
            "weibull": LAW_WEIBULL, "erlang": LAW_ERLANG}[kind]
    return Law(code, int(k), float(a), float(b))


def params(model: int, latent: Law | None, infectious: Law, beta: float, dt: float,
           seed: int, rep: int = 0, age_dtype: int = AGE_F32, shed_mode: int = SHED_NONE,
           shedding: Law | None = None) -> Params:
    """shed_mode / shedding: the shedding profile s(tau) of Eq. 8 (SHED_NONE: s = 1)."""
    return Params(model, age_dtype, latent if latent is not None else Law(0, 0, 0.0, 0.0),
                  infectious, float(beta), float(dt), int(seed), int(rep), int(shed_mode),
                  shedding if shedding is not None else Law(0, 0, 0.0, 0.0))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            u8p, f32p, f64p = P(ctypes.c_uint8), P(ctypes.c_float), P(ctypes.c_double)
            i32p, i64p, u32p = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_uint32)
            L.fso_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.fso_philox4x32_10.restype = None
            L.fso_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64]
            L.fso_uniform.restype = ctypes.c_double
            L.fso_erfcx.argtypes = [ctypes.c_double]
            L.fso_erfcx.restype = ctypes.c_double
            L.fso_hazard.argtypes = [P(Law), ctypes.c_double]
            L.fso_hazard.restype = ctypes.c_double
            L.fso_f32_to_f16_bits.argtypes = [ctypes.c_float]
            L.fso_f32_to_f16_bits.restype = ctypes.c_uint16
            L.fso_f16_bits_to_f32.argtypes = [ctypes.c_uint16]
            L.fso_f16_bits_to_f32.restype = ctypes.c_float
            L.fso_f32_to_bf16_bits.argtypes = [ctypes.c_float]
            L.fso_f32_to_bf16_bits.restype = ctypes.c_uint16
            L.fso_bf16_bits_to_f32.argtypes = [ctypes.c_uint16]
            L.fso_bf16_bits_to_f32.restype = ctypes.c_float
            L.fso_store_age.argtypes = [ctypes.c_float, ctypes.c_int32]
            L.fso_store_age.restype = ctypes.c_float
            L.fso_age_next.argtypes = [ctypes.c_float, ctypes.c_double, ctypes.c_int32]
            L.fso_age_next.restype = ctypes.c_float
            L.fso_init.argtypes = [ctypes.c_int64, i32p, ctypes.c_int64, ctypes.c_int32, u8p, f32p]
            L.fso_init.restype = ctypes.c_int
            L.fso_counts.argtypes = [ctypes.c_int64, u8p, u32p]
            L.fso_counts.restype = None
            L.fso_step.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_int64,
                                   u8p, f32p, u8p, f32p, f64p, f64p]
            L.fso_step.restype = ctypes.c_int
            L.fso_density.argtypes = [P(Law), ctypes.c_double]
            L.fso_density.restype = ctypes.c_double
            L.fso_shedding.argtypes = [P(Params), ctypes.c_double]
            L.fso_shedding.restype = ctypes.c_double
            L.fso_infectivity.argtypes = [P(Params), ctypes.c_float]
            L.fso_infectivity.restype = ctypes.c_float
            L.fso_step_rho.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_int64,
                                       u8p, f32p, f32p, u8p, f32p, f32p, f64p, f64p]
            L.fso_step_rho.restype = ctypes.c_int
            L.fso_markov_tau.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, u8p, f64p, f64p]
            L.fso_markov_tau.restype = ctypes.c_float
            L.fso_markov_step.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_float, ctypes.c_int64, u8p, f32p, u8p, f32p,
                                          f64p, f32p]
            L.fso_markov_step.restype = ctypes.c_int
            L.fso_markov_run.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, u8p, f32p,
                                         u32p, P(ctypes.c_int64)]
            L.fso_markov_run.restype = ctypes.c_int
            L.fso_gillespie_run.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), i32p, ctypes.c_int64,
                                            ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, u32p]
            L.fso_gillespie_run.restype = ctypes.c_int
            L.fso_run.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_int64,
                                  ctypes.c_int64, u8p, f32p, u32p]
            L.fso_run.restype = ctypes.c_int
            L.fso_adaptive_dt.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.fso_adaptive_dt.restype = ctypes.c_float
            L.fso_run_adaptive.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int64, ctypes.c_int64, u8p, f32p, u32p, f32p,
                                           P(ctypes.c_double)]
            L.fso_run_adaptive.restype = ctypes.c_int
            L.fso_exact_run.argtypes = [ctypes.c_int64, i64p, i32p, P(Params), i32p, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_double, u32p]
            L.fso_exact_run.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------- scalars
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().fso_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def uniform(seed: int, rep: int, step: int, node: int) -> float:
    return lib().fso_uniform(seed, rep, step, node)


def erfcx(z: float) -> float:
    return lib().fso_erfcx(z)


def hazard(lw: Law, tau: float) -> float:
    return lib().fso_hazard(ctypes.byref(lw), tau)


def store_age(x: float, age_dtype: int) -> float:
    return lib().fso_store_age(x, age_dtype)


def age_next(age: float, dt: float, age_dtype: int) -> float:
    return lib().fso_age_next(age, dt, age_dtype)


def f16_bits(x: float) -> int:
    return lib().fso_f32_to_f16_bits(x)


def bf16_bits(x: float) -> int:
    return lib().fso_f32_to_bf16_bits(x)


# ---------------------------------------------------------------- arrays
def init(n: int, index_nodes, index_state: int):
    idx = np.ascontiguousarray(index_nodes, dtype=np.int32)
    X = np.zeros(n, dtype=np.uint8)
    A = np.zeros(n, dtype=np.float32)
    rc = lib().fso_init(n, _ptr(idx, ctypes.c_int32), idx.size, index_state,
                        _ptr(X, ctypes.c_uint8), _ptr(A, ctypes.c_float))
    if rc:
        raise ValueError("oracle init rejected the index list")
    return X, A


def counts(X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.uint8)
    c = np.zeros(4, dtype=np.uint32)
    lib().fso_counts(X.size, _ptr(X, ctypes.c_uint8), _ptr(c, ctypes.c_uint32))
    return c


def step(row_ptr, col_ind, prm: Params, k: int, X, A, want_margin=False, want_lambda=False):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    A = np.ascontiguousarray(A, dtype=np.float32)
    n = X.size
    Xn = np.empty_like(X)
    An = np.empty_like(A)
    margin = np.empty(n, dtype=np.float64) if want_margin else None
    lam = np.empty(n, dtype=np.float64) if want_lambda else None
    rc = lib().fso_step(n, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm), k,
                        _ptr(X, ctypes.c_uint8), _ptr(A, ctypes.c_float),
                        _ptr(Xn, ctypes.c_uint8), _ptr(An, ctypes.c_float),
                        _ptr(margin, ctypes.c_double) if margin is not None else None,
                        _ptr(lam, ctypes.c_double) if lam is not None else None)
    if rc:
        raise ValueError("oracle step rejected the state")
    return Xn, An, margin, lam


def density(lw: Law, tau: float) -> float:
    return lib().fso_density(ctypes.byref(lw), float(tau))


def shedding(prm: Params, tau: float) -> float:
    """s(tau) of Eq. 8."""
    return lib().fso_shedding(ctypes.byref(prm), float(tau))


def infectivity(prm: Params, tau: float) -> float:
    """The stored infectivity beta s(tau) of an I node (fp32, then the storage type)."""
    return lib().fso_infectivity(ctypes.byref(prm), float(tau))


def step_rho(row_ptr, col_ind, prm: Params, k: int, X, A, rho_in=None):
    """One step with the infectivity explicit: rho_in (float32[n] as stored,
    None = computed from the ages). Returns (Xn, An, rho_next, margin, lam)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    A = np.ascontiguousarray(A, dtype=np.float32)
    rin = None if rho_in is None else np.ascontiguousarray(rho_in, dtype=np.float32)
    n = X.size
    Xn = np.empty_like(X)
    An = np.empty_like(A)
    rout = np.empty(n, dtype=np.float32)
    margin = np.empty(n, dtype=np.float64)
    lam = np.empty(n, dtype=np.float64)
    rc = lib().fso_step_rho(n, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm), k,
                            _ptr(X, ctypes.c_uint8), _ptr(A, ctypes.c_float),
                            _ptr(rin, ctypes.c_float) if rin is not None else None,
                            _ptr(Xn, ctypes.c_uint8), _ptr(An, ctypes.c_float), _ptr(rout, ctypes.c_float),
                            _ptr(margin, ctypes.c_double), _ptr(lam, ctypes.c_double))
    if rc:
        raise ValueError("oracle step rejected the state or the parameters")
    return Xn, An, rout, margin, lam


def markov_tau(row_ptr, col_ind, prm: Params, theta: float, p_max: float, tau_max: float, X):
    """Algorithm 1's step size for state X: (tau as float, Lambda, max lambda)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    lam, lmax = ctypes.c_double(), ctypes.c_double()
    tau = lib().fso_markov_tau(X.size, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm),
                               theta, p_max, tau_max, _ptr(X, ctypes.c_uint8), ctypes.byref(lam),
                               ctypes.byref(lmax))
    return tau, lam.value, lmax.value


def markov_step(row_ptr, col_ind, prm: Params, theta: float, p_max: float, tau_max: float, k: int, X, A,
                tau_in: float = 0.0):
    """One step of Algorithm 1 (tau_in > 0 overrides the rule). Returns (Xn, An, margin, tau)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    A = np.ascontiguousarray(A, dtype=np.float32)
    Xn = np.empty_like(X)
    An = np.empty_like(A)
    margin = np.empty(X.size, dtype=np.float64)
    tau = ctypes.c_float()
    rc = lib().fso_markov_step(X.size, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm),
                               theta, p_max, tau_max, float(tau_in), k, _ptr(X, ctypes.c_uint8),
                               _ptr(A, ctypes.c_float), _ptr(Xn, ctypes.c_uint8), _ptr(An, ctypes.c_float),
                               _ptr(margin, ctypes.c_double), ctypes.byref(tau))
    if rc:
        raise ValueError("oracle Markov step rejected the state or the parameters")
    return Xn, An, margin, tau.value


def markov_run(row_ptr, col_ind, prm: Params, theta: float, p_max: float, tau_max: float, k0: int,
               n_grid: int, grid_dt: float, X, A):
    """Algorithm 1 steps until t = (n_grid - 1) grid_dt; returns (counts[n_grid, 4], X, A, steps)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.array(X, dtype=np.uint8, copy=True)
    A = np.array(A, dtype=np.float32, copy=True)
    cnt = np.zeros((n_grid, 4), dtype=np.uint32)
    steps = ctypes.c_int64()
    rc = lib().fso_markov_run(X.size, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm),
                              theta, p_max, tau_max, k0, n_grid, grid_dt, _ptr(X, ctypes.c_uint8),
                              _ptr(A, ctypes.c_float), _ptr(cnt, ctypes.c_uint32), ctypes.byref(steps))
    if rc:
        raise ValueError("oracle Markov run failed")
    return cnt, X, A, steps.value


def gillespie_run(row_ptr, col_ind, prm: Params, index_nodes, index_state: int, rng_seed: int,
                  n_grid: int, grid_dt: float) -> np.ndarray:
    """Exact Doob-Gillespie run; counts[n_grid, 4] at t = g * grid_dt."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    idx = np.ascontiguousarray(index_nodes, dtype=np.int32)
    cnt = np.zeros((n_grid, 4), dtype=np.uint32)
    rc = lib().fso_gillespie_run(rp.size - 1, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32),
                                 ctypes.byref(prm), _ptr(idx, ctypes.c_int32), idx.size, index_state, rng_seed,
                                 n_grid, grid_dt, _ptr(cnt, ctypes.c_uint32))
    if rc:
        raise ValueError("Gillespie run failed")
    return cnt


def run(row_ptr, col_ind, prm: Params, k0: int, steps: int, X, A):
    """Returns (counts[(steps+1), 4], X, A) after `steps` steps from k0."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.array(X, dtype=np.uint8, copy=True)
    A = np.array(A, dtype=np.float32, copy=True)
    cnt = np.zeros((steps + 1, 4), dtype=np.uint32)
    rc = lib().fso_run(X.size, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm),
                       k0, steps, _ptr(X, ctypes.c_uint8), _ptr(A, ctypes.c_float),
                       _ptr(cnt, ctypes.c_uint32))
    if rc:
        raise ValueError("oracle run failed")
    return cnt, X, A


def adaptive_dt(dt_max: float, eps: float, delta: float, lambda_prev: float) -> float:
    """Section 5.2: min(dt_max, eps / (lambda_prev + delta)) as the float ages advance by."""
    return lib().fso_adaptive_dt(dt_max, eps, delta, lambda_prev)


def run_adaptive(row_ptr, col_ind, prm: Params, eps: float, delta: float, k0: int, steps: int, X, A,
                 lambda_prev: float = 0.0):
    """Adaptive steps (prm.dt = dt_max). Returns (counts[(steps+1), 4], X, A,
    dts[steps], lambda of the last step's largest rate)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    X = np.array(X, dtype=np.uint8, copy=True)
    A = np.array(A, dtype=np.float32, copy=True)
    cnt = np.zeros((steps + 1, 4), dtype=np.uint32)
    dts = np.zeros(steps, dtype=np.float32)
    last = ctypes.c_double(0.0)
    rc = lib().fso_run_adaptive(X.size, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm),
                                eps, delta, lambda_prev, k0, steps, _ptr(X, ctypes.c_uint8),
                                _ptr(A, ctypes.c_float), _ptr(cnt, ctypes.c_uint32), _ptr(dts, ctypes.c_float),
                                ctypes.byref(last))
    if rc:
        raise ValueError("oracle adaptive run failed")
    return cnt, X, A, dts, last.value


def exact_run(row_ptr, col_ind, prm: Params, index_nodes, index_state: int, rng_seed: int,
              n_grid: int, grid_dt: float) -> np.ndarray:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_ind, dtype=np.int32)
    idx = np.ascontiguousarray(index_nodes, dtype=np.int32)
    n = rp.size - 1
    out = np.zeros((n_grid, 4), dtype=np.uint32)
    rc = lib().fso_exact_run(n, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), ctypes.byref(prm),
                             _ptr(idx, ctypes.c_int32), idx.size, index_state, rng_seed,
                             n_grid, grid_dt, _ptr(out, ctypes.c_uint32))
    if rc:
        raise ValueError("exact simulator failed")
    return out
