"""Python binding of the swept-rule CUDA library (``include/swept.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  The functions keep the
C names; errors raise ``SweptError`` with the library's message.  The
library must have been built (``python -m paper_1504_01380_gb300.build``);
nothing here falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libswept.so")

SWEPT_F64, SWEPT_F32C, SWEPT_F32 = 0, 1, 2
SWEPT_HEAT, SWEPT_KS, SWEPT_HEAT_RK2, SWEPT_KS_RK2, SWEPT_EULER = 0, 1, 2, 3, 4
SWEPT_SUM, SWEPT_HALF_SUMSQ, SWEPT_DOT = 0, 1, 2
SWEPT_OK, SWEPT_EINVAL, SWEPT_ENOMEM, SWEPT_ECUDA, SWEPT_ETIMEOUT, SWEPT_ENOTSUP = 0, -1, -2, -3, -4, -5
SWEPT_ETOOBIG = -6
SWEPT_NOALLOC_MAX_N = 1 << 20
SWEPT_OPT_DIAMOND, SWEPT_OPT_RING_WARPS, SWEPT_OPT_GRAPH, SWEPT_OPT_PDL, SWEPT_OPT_PERSISTENT = 0, 1, 2, 3, 4
SWEPT_OPT_DROP_WINDOW, SWEPT_OPT_TIMEOUT_MS, SWEPT_OPT_STREAM, SWEPT_OPT_TIME_RING = 5, 6, 7, 8
SWEPT_OPT_RESIDENT, SWEPT_OPT_NAIVE_RESIDENT = 9, 10
SWEPT_DIAMOND_AUTO, SWEPT_DIAMOND_WINDOW, SWEPT_DIAMOND_RING = 0, 1, 2
SWEPT_PROBE_F32_ADD, SWEPT_PROBE_F32_FMA, SWEPT_PROBE_F64_ADD, SWEPT_PROBE_F64_FMA = 0, 1, 2, 3

RADIUS = {SWEPT_HEAT: 1, SWEPT_KS: 2, SWEPT_HEAT_RK2: 1, SWEPT_KS_RK2: 2, SWEPT_EULER: 1}

# Every entry point declared in include/swept.h.
EXPORTS = (
    "swept_plan", "swept_destroy", "swept_plan_info", "swept_advance", "swept_naive_advance",
    "swept_f32c_split", "swept_f32c_merge", "swept_reduce", "swept_strerror", "swept_version",
    "swept_advance_noalloc", "swept_plan_set",
    "swept_batch_plan", "swept_batch_set", "swept_batch_info", "swept_advance_batch",
    "swept_batch_status", "swept_batch_destroy", "swept_adjoint", "swept_batch_naive_advance",
    "swept_plan_status", "swept_plan_last_advance", "swept_probe_alu", "swept_adjoint_scratch",
    "swept_check_div_sqrt",
    "swept_stage", "swept_edge_copy",
)

SWEPT_BOPT_TIMEOUT_S, SWEPT_BOPT_DROP_ITEM, SWEPT_BOPT_GRID, SWEPT_BOPT_GRAPH, SWEPT_BOPT_RUN_LEN = 0, 1, 2, 3, 4


class swept_problem_t(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nsteps", ctypes.c_int64), ("offset", ctypes.c_int64),
                ("stencil", ctypes.c_int), ("reserved", ctypes.c_int),
                ("params", ctypes.c_double * 2)]

_lock = threading.Lock()
_lib = None


class SweptError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


def load(path: str | None = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"swept CUDA library not built: {p} is missing "
                               "(run python -m paper_1504_01380_gb300.build)")
        L = ctypes.CDLL(p)
        vp, i64, i32, dbl_p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.swept_plan.argtypes = [ctypes.POINTER(vp), i64, i32, i32, ctypes.POINTER(ctypes.c_double),
                                 i32, i32, i32]
        L.swept_plan.restype = i32
        L.swept_destroy.argtypes = [vp]
        L.swept_destroy.restype = None
        L.swept_plan_info.argtypes = [vp, ctypes.POINTER(i64), i32]
        L.swept_plan_info.restype = i32
        L.swept_plan_set.argtypes = [vp, i32, i64]
        L.swept_plan_set.restype = i32
        for f in ("swept_advance", "swept_naive_advance"):
            getattr(L, f).argtypes = [vp, vp, i64, vp]
            getattr(L, f).restype = i32
        L.swept_f32c_split.argtypes = [i64, vp, vp, vp]
        L.swept_f32c_split.restype = i32
        L.swept_f32c_merge.argtypes = [i64, vp, vp, vp]
        L.swept_f32c_merge.restype = i32
        L.swept_reduce.argtypes = [vp, vp, i32, vp, dbl_p, vp]
        L.swept_reduce.restype = i32
        L.swept_advance_noalloc.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_double), i32, i32, i32,
                                            vp, i64, vp]
        L.swept_advance_noalloc.restype = i32
        L.swept_batch_plan.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(swept_problem_t), i32, i32, i32]
        L.swept_batch_plan.restype = i32
        L.swept_batch_set.argtypes = [vp, i32, ctypes.c_double]
        L.swept_batch_set.restype = i32
        L.swept_batch_info.argtypes = [vp, ctypes.POINTER(i64), i32]
        L.swept_batch_info.restype = i32
        L.swept_advance_batch.argtypes = [vp, vp, vp]
        L.swept_advance_batch.restype = i32
        L.swept_batch_naive_advance.argtypes = [vp, vp, vp]
        L.swept_batch_naive_advance.restype = i32
        L.swept_plan_status.argtypes = [vp, vp]
        L.swept_plan_status.restype = i32
        L.swept_plan_last_advance.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                              ctypes.POINTER(ctypes.c_double)]
        L.swept_plan_last_advance.restype = i32
        L.swept_batch_status.argtypes = [vp, vp]
        L.swept_batch_status.restype = i32
        L.swept_batch_destroy.argtypes = [vp]
        L.swept_batch_destroy.restype = None
        L.swept_adjoint.argtypes = [vp, vp, vp, vp, i64, i32, vp]
        L.swept_adjoint.restype = i32
        L.swept_stage.argtypes = [vp, vp, i64, i32, i32, vp]
        L.swept_stage.restype = i32
        L.swept_edge_copy.argtypes = [vp, i64, i32, i32, vp, i32, vp]
        L.swept_edge_copy.restype = i32
        L.swept_adjoint_scratch.argtypes = [vp, i64, i32, ctypes.POINTER(i64)]
        L.swept_adjoint_scratch.restype = i32
        L.swept_probe_alu.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_double), vp]
        L.swept_probe_alu.restype = i32
        L.swept_check_div_sqrt.argtypes = [vp, vp, i64, vp, vp, vp]
        L.swept_check_div_sqrt.restype = i32
        L.swept_strerror.argtypes = [i32]
        L.swept_strerror.restype = ctypes.c_char_p
        L.swept_version.argtypes = []
        L.swept_version.restype = ctypes.c_char_p
        _lib = L
        return _lib


def strerror(code: int) -> str:
    return load().swept_strerror(int(code)).decode()


def swept_version() -> str:
    return load().swept_version().decode()


def _check(rc: int, what: str):
    if rc != SWEPT_OK:
        raise SweptError(rc, what)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, nbytes: int, what: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{what}: tensor is on {t.device}, but the current device is "
                         f"cuda:{torch.cuda.current_device()} (the library runs every call there)")
    if t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{what}: tensor holds {t.numel() * t.element_size()} bytes, needs {nbytes}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A validated problem with its device scratch (``swept_plan`` / ``swept_destroy``)."""

    def __init__(self, handle, N, stencil, dtype, B, H, params):
        self._h = handle
        self.N, self.stencil, self.dtype, self.B, self.h = N, stencil, dtype, B, H
        self.radius = RADIUS[stencil]
        self.params = tuple(params)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("plan was destroyed")
        return self._h

    @property
    def state_bytes(self) -> int:
        if self.stencil == SWEPT_EULER:
            return 24 * self.N
        return (4 if self.dtype == SWEPT_F32 else 8) * self.N

    def destroy(self):
        if self._h is not None:
            load().swept_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def swept_plan(N: int, radius: int, stencil_id: int, params, dtype: int, B: int = 0) -> Plan:
    L = load()
    prm = (ctypes.c_double * len(params))(*[float(x) for x in params])
    h = ctypes.c_void_p()
    _check(L.swept_plan(ctypes.byref(h), int(N), int(radius), int(stencil_id), prm, len(params),
                        int(dtype), int(B)), "swept_plan")
    info = (ctypes.c_int64 * 6)()
    _check(L.swept_plan_info(h, info, 6), "swept_plan_info")
    return Plan(h, int(N), int(stencil_id), int(dtype), int(info[0]), int(info[1]), params)


def swept_plan_set(plan: Plan, option: int, value: int) -> Plan:
    """Set a tuning option (SWEPT_OPT_*) of the plan; results do not depend on it."""
    _check(load().swept_plan_set(plan.handle, int(option), int(value)), "swept_plan_set")
    return plan


def swept_advance(plan: Plan, u, nsteps: int, stream=None):
    """u <- u after nsteps time steps (swept rule), in place on ``stream``.

    A time step is one sub-timestep for the forward-Euler stencils, two for the
    Runge-Kutta ones and four for the Euler equations (state: rho, m, E blocks).
    """
    _check(load().swept_advance(plan.handle, _dev_ptr(u, plan.state_bytes, "u"), int(nsteps),
                                _stream(stream)), "swept_advance")
    return u


def swept_plan_status(plan: Plan, stream=None) -> int:
    """Synchronise and return the device status of the last persistent or streamed advance
    (0 or SWEPT_ETIMEOUT)."""
    return int(load().swept_plan_status(plan.handle, _stream(stream)))


def swept_plan_last_advance(plan: Plan):
    """(kernel launches, ring launches, ring milliseconds or -1) of the plan's last advance;
    the time needs SWEPT_OPT_TIME_RING and waits for the advance's ring launches."""
    n, nr, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(load().swept_plan_last_advance(plan.handle, ctypes.byref(n), ctypes.byref(nr), ctypes.byref(ms)),
           "swept_plan_last_advance")
    return int(n.value), int(nr.value), float(ms.value)


def swept_stage(plan: Plan, u, k: int, hv: int, ht: int, stream=None):
    """Stage k of the swept schedule (V-fill hv, then trapezoid ht) on every window of the plan."""
    _check(load().swept_stage(plan.handle, _dev_ptr(u, plan.state_bytes, "u"), int(k), int(hv), int(ht),
                              _stream(stream)), "swept_stage")
    return u


def edge_element_bytes(plan: Plan) -> int:
    """Bytes of one leading-edge element of the plan (what swept_edge_copy moves B of)."""
    if plan.stencil == SWEPT_EULER:
        return 72 if plan.dtype == SWEPT_F64 else 48
    if plan.stencil in (SWEPT_HEAT_RK2, SWEPT_KS_RK2):
        return 16
    return 4 if plan.dtype == SWEPT_F32 else 8


def swept_edge_copy(plan: Plan, k: int, window: int, side: int, buf, to_plan: bool, stream=None):
    """Copy window's left (side 0) or right (side 1) edge half of stage k's edge buffer into buf,
    or (to_plan) from buf into the plan."""
    _check(load().swept_edge_copy(plan.handle, int(k), int(window), int(side),
                                  _dev_ptr(buf, plan.B * edge_element_bytes(plan), "buf"), 1 if to_plan else 0,
                                  _stream(stream)), "swept_edge_copy")
    return buf


def swept_naive_advance(plan: Plan, u, nsteps: int, stream=None):
    """Same result by per-step stepping (one launch per sub-timestep)."""
    _check(load().swept_naive_advance(plan.handle, _dev_ptr(u, plan.state_bytes, "u"), int(nsteps),
                                      _stream(stream)), "swept_naive_advance")
    return u


def swept_f32c_split(u64, out=None, stream=None):
    """FP64 tensor -> compensated FP32 state tensor (hi then lo, float32[2N])."""
    import torch
    n = u64.numel()
    if u64.dtype != torch.float64:
        raise TypeError("swept_f32c_split: expected float64")
    if out is None:
        out = torch.empty(2 * n, dtype=torch.float32, device=u64.device)
    _check(load().swept_f32c_split(n, _dev_ptr(u64, 8 * n, "u64"), _dev_ptr(out, 8 * n, "u32c"),
                                   _stream(stream)), "swept_f32c_split")
    return out


def swept_f32c_merge(u32c, out=None, stream=None):
    """Compensated FP32 state tensor -> FP64 tensor of hi + lo."""
    import torch
    n = u32c.numel() // 2
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=u32c.device)
    _check(load().swept_f32c_merge(n, _dev_ptr(u32c, 8 * n, "u32c"), _dev_ptr(out, 8 * n, "u64"),
                                   _stream(stream)), "swept_f32c_merge")
    return out


def swept_reduce(plan: Plan, u, what: int, v=None, out=None, stream=None):
    """FP64 reduction of the state into a 1-element device tensor (no host sync)."""
    import torch
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=u.device)
    vp = _dev_ptr(v, 8 * plan.N, "v") if v is not None else ctypes.c_void_p(0)
    _check(load().swept_reduce(plan.handle, _dev_ptr(u, (4 if plan.dtype == SWEPT_F32 else 8) * plan.N, "u"),
                               int(what), vp,
                               _dev_ptr(out, 8, "out"), _stream(stream)), "swept_reduce")
    return out


def swept_probe_alu(kind: int, iters: int, stream=None) -> float:
    """Enqueue the peak-rate probe (SWEPT_PROBE_*) on ``stream``; returns the operations it
    performs (time it with CUDA events on the same stream)."""
    ops = ctypes.c_double()
    _check(load().swept_probe_alu(int(kind), int(iters), ctypes.byref(ops), _stream(stream)),
           "swept_probe_alu")
    return float(ops.value)


def swept_check_div_sqrt(a, b, stream=None):
    """The Euler kernels' straight-line binary32 division and square root beside CUDA's
    correctly rounded ones on float32 device tensors ``a``, ``b`` (same length n).
    Returns (out, ok): out[0] the straight-line a / b, out[1] __fdiv_rn(a, b), out[2] the
    straight-line sqrt(a), out[3] __fsqrt_rn(a); ok[0] / ok[1] are 1 where the division /
    square root was proven correctly rounded (the kernels recompute the rest)."""
    import torch
    n = a.numel()
    if b.numel() != n or a.dtype != torch.float32 or b.dtype != torch.float32:
        raise ValueError("a and b must be float32 tensors of one length")
    out = torch.empty((4, n), dtype=torch.float32, device=a.device)
    ok = torch.empty((2, n), dtype=torch.int32, device=a.device)
    _check(load().swept_check_div_sqrt(_dev_ptr(a, 4 * n, "a"), _dev_ptr(b, 4 * n, "b"), int(n),
                                       _dev_ptr(out, 16 * n, "out"), _dev_ptr(ok, 8 * n, "ok"),
                                       _stream(stream)), "swept_check_div_sqrt")
    return out, ok


def swept_advance_noalloc(N: int, stencil_id: int, params, dtype: int, B: int, u, nsteps: int,
                          stream=None):
    """swept_advance without a plan and without any device allocation.

    For callers that may not allocate device memory (a fixed memory budget
    handed out by a host application, or code that must avoid the
    synchronisation an allocation can cause).  The edge scratch lives in a
    fixed 32 MiB array inside the library, so N is limited to
    SWEPT_NOALLOC_MAX_N and concurrent calls on different streams race.
    """
    prm = (ctypes.c_double * len(params))(*[float(x) for x in params])
    _check(load().swept_advance_noalloc(int(N), int(stencil_id), prm, len(params), int(dtype), int(B),
                                        _dev_ptr(u, 8 * int(N), "u"), int(nsteps), _stream(stream)),
           "swept_advance_noalloc")
    return u


class Batch:
    """A planned batch (``swept_batch_plan`` / ``swept_batch_destroy``).

    ``offsets[i]`` is the byte offset of problem i's state in the pool and
    ``pool_bytes`` the pool size, both chosen by ``swept_batch_plan`` when
    the caller does not give offsets.
    """

    def __init__(self, handle, offsets, pool_bytes, sizes, dtype):
        self._h = handle
        self.offsets, self.pool_bytes, self.sizes, self.dtype = offsets, pool_bytes, sizes, dtype

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch was destroyed")
        return self._h

    def info(self) -> dict:
        v = (ctypes.c_int64 * 6)()
        _check(load().swept_batch_info(self.handle, v, 6), "swept_batch_info")
        return {"items": v[0], "stages": v[1], "windows": v[2], "grid": v[3], "problems": v[4],
                "run_len": v[5]}

    def destroy(self):
        if self._h is not None:
            load().swept_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def swept_batch_plan(problems, dtype: int, B_heat: int = 0, B_ks: int = 0, offsets=None) -> Batch:
    """problems: iterable of (stencil, N, nsteps, params).  Offsets default to a packed pool."""
    problems = list(problems)
    arr = (swept_problem_t * len(problems))()
    offs, pos = [], 0
    for i, (stencil, n, nsteps, params) in enumerate(problems):
        off = offsets[i] if offsets is not None else pos
        pos = max(pos, off + 8 * int(n))
        pos = (pos + 255) // 256 * 256
        prm = list(params) + [0.0] * (2 - len(params))
        arr[i] = swept_problem_t(int(n), int(nsteps), int(off), int(stencil), 0,
                                 (ctypes.c_double * 2)(*prm))
        offs.append(int(off))
    h = ctypes.c_void_p()
    _check(load().swept_batch_plan(ctypes.byref(h), len(problems), arr, int(dtype), int(B_heat), int(B_ks)),
           "swept_batch_plan")
    return Batch(h, offs, pos, [int(p[1]) for p in problems], int(dtype))


def swept_batch_set(batch: Batch, option: int, value: float) -> Batch:
    _check(load().swept_batch_set(batch.handle, int(option), float(value)), "swept_batch_set")
    return batch


def swept_advance_batch(batch: Batch, pool, stream=None):
    """Advance every problem of the batch in ``pool`` (a CUDA tensor of pool_bytes bytes)."""
    _check(load().swept_advance_batch(batch.handle, _dev_ptr(pool, batch.pool_bytes, "pool"),
                                      _stream(stream)), "swept_advance_batch")
    return pool


def swept_batch_naive_advance(batch: Batch, pool, stream=None):
    """Same result by one launch per time step over the problems still active (baseline)."""
    _check(load().swept_batch_naive_advance(batch.handle, _dev_ptr(pool, batch.pool_bytes, "pool"),
                                            _stream(stream)), "swept_batch_naive_advance")
    return pool


def swept_batch_status(batch: Batch, stream=None) -> int:
    """Synchronise and return the device status of the last advance (0 or SWEPT_ETIMEOUT)."""
    return int(load().swept_batch_status(batch.handle, _stream(stream)))


def swept_adjoint(plan: Plan, u0, lam_T, nsteps: int, K_cycles: int = 64, out=None, stream=None):
    """(d u(nsteps)/d u0)^T lam_T for an FP64 plan; lam_T = u(nsteps) gives grad of 1/2 sum u^2."""
    import torch
    if out is None:
        out = torch.empty_like(u0)
    _check(load().swept_adjoint(plan.handle, _dev_ptr(u0, plan.state_bytes, "u0"),
                                _dev_ptr(lam_T, plan.state_bytes, "lam_T"),
                                _dev_ptr(out, plan.state_bytes, "grad"), int(nsteps), int(K_cycles),
                                _stream(stream)), "swept_adjoint")
    return out


def swept_adjoint_scratch(plan: Plan, nsteps: int, K_cycles: int = 64) -> int:
    """Device bytes swept_adjoint allocates for this plan, step count and checkpoint bound."""
    b = ctypes.c_int64()
    _check(load().swept_adjoint_scratch(plan.handle, int(nsteps), int(K_cycles), ctypes.byref(b)),
           "swept_adjoint_scratch")
    return int(b.value)


def _make_autograd():
    import torch

    class SweptAdvance(torch.autograd.Function):
        """u(nsteps) = swept advance of u0; backward runs the swept adjoint."""

        @staticmethod
        def forward(ctx, u0, plan, nsteps, K_cycles=64):
            u = u0.detach().clone().contiguous()
            swept_advance(plan, u, nsteps)
            ctx.save_for_backward(u0.detach().contiguous())
            ctx.plan, ctx.nsteps, ctx.K = plan, int(nsteps), int(K_cycles)
            return u

        @staticmethod
        def backward(ctx, grad_out):
            (u0,) = ctx.saved_tensors
            g = swept_adjoint(ctx.plan, u0, grad_out.contiguous(), ctx.nsteps, ctx.K)
            return g, None, None, None

    return SweptAdvance


def __getattr__(name):
    if name == "SweptAdvance":
        cls = _make_autograd()
        globals()["SweptAdvance"] = cls
        return cls
    raise AttributeError(name)
