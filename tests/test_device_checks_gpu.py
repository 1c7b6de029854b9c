"""Every entry point refuses memory that is not on the current device before it launches anything.

A kernel given a pointer it cannot reach faults the GPU, so the C ABI checks the
pointers (and the stream and the plan's device) first.  With one GPU the foreign
memory here is host memory: pinned (a registered host pointer) and pageable (an
unregistered one).  The calls go straight through ctypes, past the Python
wrapper's own check, and must return SWEPT_EINVAL with nothing enqueued; the next
call with device memory is exact.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from tests.test_parity_gpu import assert_same, initial, oracle_run, params_of, run_gpu

pytestmark = pytest.mark.gpu


def _host_pointers(nbytes):
    import torch
    pinned = torch.zeros(nbytes // 8, dtype=torch.float64).pin_memory()
    pageable = np.zeros(nbytes // 8)
    return [(pinned, ctypes.c_void_p(pinned.data_ptr())),
            (pageable, ctypes.c_void_p(pageable.ctypes.data))]


def test_host_memory_is_refused(cuda_lib):
    import torch
    sw = cuda_lib
    L = sw.load()
    N, B = 8 * 128, 128
    plan = sw.swept_plan(N, 1, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F64, B)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dev = torch.zeros(N, dtype=torch.float64, device="cuda")
    out1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for keep, hp in _host_pointers(8 * N):
        assert L.swept_advance(plan.handle, hp, 10, stream) == sw.SWEPT_EINVAL
        assert L.swept_naive_advance(plan.handle, hp, 10, stream) == sw.SWEPT_EINVAL
        assert L.swept_reduce(plan.handle, hp, sw.SWEPT_SUM, None,
                              ctypes.c_void_p(out1.data_ptr()), stream) == sw.SWEPT_EINVAL
        assert L.swept_reduce(plan.handle, ctypes.c_void_p(dev.data_ptr()), sw.SWEPT_SUM, None,
                              hp, stream) == sw.SWEPT_EINVAL
        assert L.swept_adjoint(plan.handle, hp, ctypes.c_void_p(dev.data_ptr()),
                               ctypes.c_void_p(dev.data_ptr()), 10, 0, stream) == sw.SWEPT_EINVAL
        assert L.swept_f32c_split(N, hp, ctypes.c_void_p(dev.data_ptr()), stream) == sw.SWEPT_EINVAL
        assert L.swept_f32c_merge(N // 2, ctypes.c_void_p(dev.data_ptr()), hp, stream) == sw.SWEPT_EINVAL
        prm = (ctypes.c_double * 1)(0.25)
        assert L.swept_advance_noalloc(N, sw.SWEPT_HEAT, prm, 1, sw.SWEPT_F64, B, hp, 10,
                                       stream) == sw.SWEPT_EINVAL
    torch.cuda.synchronize()
    # the context is untouched: the same plan on device memory is exact
    u0 = initial(0, N, 3)
    assert_same(plan, run_gpu(sw, plan, u0, 100), oracle_run(0, sw.SWEPT_F64, u0, 100))
    plan.destroy()


def test_batch_refuses_host_pool(cuda_lib):
    import torch
    sw = cuda_lib
    L = sw.load()
    batch = sw.swept_batch_plan([(0, 1024, 50, (0.25,)), (1, 2048, 40, params_of(1))], sw.SWEPT_F32C,
                                256, 256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for keep, hp in _host_pointers(batch.pool_bytes + 64):
        assert L.swept_advance_batch(batch.handle, hp, stream) == sw.SWEPT_EINVAL
        assert L.swept_batch_naive_advance(batch.handle, hp, stream) == sw.SWEPT_EINVAL
    torch.cuda.synchronize()
    batch.destroy()


def test_python_wrapper_names_the_device(cuda_lib):
    import torch
    sw = cuda_lib
    plan = sw.swept_plan(256, 1, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F64, 64)
    with pytest.raises(TypeError):
        sw.swept_advance(plan, torch.zeros(256, dtype=torch.float64), 5)      # a CPU tensor
    plan.destroy()
