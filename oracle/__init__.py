"""CPU oracle for the swept-rule hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports it, and
this package imports nothing from the product path.

Contents
--------
* ``oracle.c`` (compiled here with gcc): per-step FP64, plain FP32 and
  FP32-compensated steppers, split/merge of the compensated state, the discrete adjoint, the
  two-stage Runge-Kutta steppers and the Euler-equations finite-volume
  scheme (Section 7: second-order reconstruction with minmod, Roe spectral
  radius dissipation, midpoint rule; four sub-timesteps per time step), in
  FP64 and on the compensated FP32 state (binary32 fluxes, TwoSum update).
  These follow the definition the swept rule reorders (Sections 2-3): one
  sub-timestep applied to every point of the periodic grid, level after level.
* ``pointwise.py``: the same sub-timestep for a single point in Python, with
  a correctly rounded fma, used by the swept brute force.
* ``swept_bruteforce.py``: a literal simulation of the paper's swept stages
  (Section 3) on tiny grids.
* ``reductions.py``: exactly rounded sums for the conserved-sum, objective
  and directional-derivative reductions.

The evaluation order of every expression is stated in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

HEAT = 0
KS = 1
HEAT_RK2 = 2
KS_RK2 = 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, no fp contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32 = ctypes.c_int64, ctypes.c_int
            dp, fp = ctypes.c_void_p, ctypes.c_void_p
            L.oracle_step_f64.argtypes = [i32, dp, dp, dp, i64]
            L.oracle_advance_f64.argtypes = [i32, dp, dp, i64, i64, i32]
            L.oracle_split_f32c.argtypes = [dp, fp, fp, i64]
            L.oracle_merge_f32c.argtypes = [fp, fp, dp, i64]
            L.oracle_step_f32c.argtypes = [i32, dp, fp, fp, fp, fp, i64]
            L.oracle_advance_f32c.argtypes = [i32, dp, fp, fp, i64, i64, i32]
            L.oracle_adjoint_f64.argtypes = [i32, dp, dp, dp, dp, i64, i64]
            L.oracle_adjoint_step_f64.argtypes = [i32, dp, dp, dp, dp, i64]
            L.oracle_advance_rk2_f64.argtypes = [i32, dp, dp, i64, i64, i32]
            L.oracle_rk2_substep_f64.argtypes = [i32, dp, i32, dp, dp, dp, i64]
            L.oracle_euler_advance.argtypes = [dp, dp, i64, i64]
            L.oracle_euler_advance_f32c.argtypes = [dp, fp, fp, i64, i64]
            L.oracle_step_f32.argtypes = [i32, dp, fp, fp, i64]
            L.oracle_advance_f32.argtypes = [i32, dp, fp, i64, i64, i32]
            for f in ("oracle_step_f64", "oracle_advance_f64", "oracle_split_f32c",
                      "oracle_merge_f32c", "oracle_step_f32c", "oracle_advance_f32c",
                      "oracle_adjoint_f64", "oracle_adjoint_step_f64", "oracle_max_threads",
                      "oracle_advance_rk2_f64", "oracle_rk2_substep_f64", "oracle_euler_advance",
                      "oracle_euler_advance_f32c", "oracle_step_f32", "oracle_advance_f32"):
                getattr(L, f).restype = i32
            _lib = L
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _params(stencil: int, params) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    need = 1 if stencil in (HEAT, HEAT_RK2) else 2
    if p.size != need:
        raise ValueError(f"stencil {stencil} takes {need} parameter(s), got {p.size}")
    return p


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def radius(stencil: int) -> int:
    return 1 if stencil in (HEAT, HEAT_RK2) else 2


def step_f64(stencil: int, params, u: np.ndarray) -> np.ndarray:
    """One sub-timestep of the FP64 scheme on the periodic array ``u``."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    p = _params(stencil, params)
    _check(lib().oracle_step_f64(stencil, _ptr(p), _ptr(u), _ptr(out), u.size), "step_f64")
    return out


def advance_f64(stencil: int, params, u: np.ndarray, nsteps: int, threads: int = 0) -> np.ndarray:
    """``nsteps`` FP64 sub-timesteps (returns a new array)."""
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    p = _params(stencil, params)
    _check(lib().oracle_advance_f64(stencil, _ptr(p), _ptr(u), u.size, int(nsteps), int(threads)),
           "advance_f64")
    return u


def step_f32(stencil: int, params, u: np.ndarray) -> np.ndarray:
    """One sub-timestep of the plain binary32 scheme (the FP64 expressions in binary32)."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    p = _params(stencil, params)
    _check(lib().oracle_step_f32(stencil, _ptr(p), _ptr(u), _ptr(out), u.size), "step_f32")
    return out


def advance_f32(stencil: int, params, u: np.ndarray, nsteps: int, threads: int = 0) -> np.ndarray:
    """``nsteps`` plain binary32 sub-timesteps (returns a new float32 array)."""
    u = np.array(u, dtype=np.float32, copy=True, order="C")
    p = _params(stencil, params)
    _check(lib().oracle_advance_f32(stencil, _ptr(p), _ptr(u), u.size, int(nsteps), int(threads)),
           "advance_f32")
    return u


def split_f32c(u: np.ndarray):
    """FP64 -> compensated pair (hi, lo): hi = fl32(u), lo = fl32(u - hi)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    hi = np.empty(u.size, dtype=np.float32)
    lo = np.empty(u.size, dtype=np.float32)
    _check(lib().oracle_split_f32c(_ptr(u), _ptr(hi), _ptr(lo), u.size), "split_f32c")
    return hi, lo


def merge_f32c(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    """Compensated pair -> FP64 value hi + lo (one FP64 rounding)."""
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    u = np.empty(hi.size, dtype=np.float64)
    _check(lib().oracle_merge_f32c(_ptr(hi), _ptr(lo), _ptr(u), hi.size), "merge_f32c")
    return u


def step_f32c(stencil: int, params, hi: np.ndarray, lo: np.ndarray):
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    ho, lout = np.empty_like(hi), np.empty_like(lo)
    p = _params(stencil, params)
    _check(lib().oracle_step_f32c(stencil, _ptr(p), _ptr(hi), _ptr(lo), _ptr(ho), _ptr(lout),
                                  hi.size), "step_f32c")
    return ho, lout


def advance_f32c(stencil: int, params, hi: np.ndarray, lo: np.ndarray, nsteps: int,
                 threads: int = 0):
    """``nsteps`` compensated-FP32 sub-timesteps on (hi, lo) (returns new arrays)."""
    hi = np.array(hi, dtype=np.float32, copy=True, order="C")
    lo = np.array(lo, dtype=np.float32, copy=True, order="C")
    p = _params(stencil, params)
    _check(lib().oracle_advance_f32c(stencil, _ptr(p), _ptr(hi), _ptr(lo), hi.size, int(nsteps),
                                     int(threads)), "advance_f32c")
    return hi, lo


def adjoint_f64(stencil: int, params, u0: np.ndarray, lam_T: np.ndarray, nsteps: int) -> np.ndarray:
    """Gradient of <lam_T, u(nsteps)> with respect to u0 (discrete adjoint, small cases)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    lam = np.ascontiguousarray(lam_T, dtype=np.float64)
    g = np.empty_like(u0)
    p = _params(stencil, params)
    _check(lib().oracle_adjoint_f64(stencil, _ptr(p), _ptr(u0), _ptr(lam), _ptr(g), u0.size,
                                    int(nsteps)), "adjoint_f64")
    return g


def adjoint_step_f64(stencil: int, params, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """(dPhi/du at u)^T lam for one sub-timestep."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.empty_like(u)
    p = _params(stencil, params)
    _check(lib().oracle_adjoint_step_f64(stencil, _ptr(p), _ptr(u), _ptr(lam), _ptr(out), u.size),
           "adjoint_step_f64")
    return out


def advance_rk2_f64(stencil: int, params, u: np.ndarray, nsteps: int, threads: int = 0) -> np.ndarray:
    """``nsteps`` two-stage Runge-Kutta (midpoint) time steps = 2*nsteps sub-timesteps."""
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    p = _params(stencil, params)
    _check(lib().oracle_advance_rk2_f64(stencil, _ptr(p), _ptr(u), u.size, int(nsteps), int(threads)),
           "advance_rk2_f64")
    return u


def rk2_substep_f64(stencil: int, params, sub: int, u: np.ndarray, m: np.ndarray | None = None) -> np.ndarray:
    """Sub-timestep A (sub=0: midpoint from u) or B (sub=1: next u from u and the midpoint m)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    m = u if m is None else np.ascontiguousarray(m, dtype=np.float64)
    out = np.empty_like(u)
    p = _params(stencil, params)
    _check(lib().oracle_rk2_substep_f64(stencil, _ptr(p), int(sub), _ptr(u), _ptr(m), _ptr(out), u.size),
           "rk2_substep_f64")
    return out


def euler_advance(params, q: np.ndarray, nsteps: int) -> np.ndarray:
    """Euler equations (rho, m, E), shape (N, 3): nsteps RK2 steps of 4 sub-timesteps."""
    q = np.array(q, dtype=np.float64, copy=True, order="C")
    if q.ndim != 2 or q.shape[1] != 3:
        raise ValueError("q must have shape (N, 3)")
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if p.size != 3:
        raise ValueError("Euler takes (dt, dx, gamma)")
    _check(lib().oracle_euler_advance(_ptr(p), _ptr(q), q.shape[0], int(nsteps)), "euler_advance")
    return q


def euler_advance_f32c(params, hi: np.ndarray, lo: np.ndarray, nsteps: int):
    """Euler equations on the compensated state (hi, lo), each of shape (N, 3) float32."""
    hi = np.array(hi, dtype=np.float32, copy=True, order="C")
    lo = np.array(lo, dtype=np.float32, copy=True, order="C")
    if hi.ndim != 2 or hi.shape[1] != 3 or lo.shape != hi.shape:
        raise ValueError("hi and lo must have shape (N, 3)")
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if p.size != 3:
        raise ValueError("Euler takes (dt, dx, gamma)")
    _check(lib().oracle_euler_advance_f32c(_ptr(p), _ptr(hi), _ptr(lo), hi.shape[0], int(nsteps)),
           "euler_advance_f32c")
    return hi, lo


def max_threads() -> int:
    return int(lib().oracle_max_threads())
