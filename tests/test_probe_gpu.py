"""The peak-rate probe: its FP32 rate sits just under the SM-count x lanes x clock ceiling.

The probe is the roofline denominator of the swept kernels, so it must measure
the pipe and nothing else: a rate above 152 SMs x 128 FP32 lanes x the maximum
SM clock would mean the work was not done, one far below it that the chains do
not fill the pipe.  FP64 must be slower than FP32 (GB300's FP64 pipe is narrow)
and adds and fmas count one operation each.
"""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu


def _rate(sw, kind, iters):
    import torch
    ops = sw.swept_probe_alu(kind, iters)            # warm-up launch
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ops = sw.swept_probe_alu(kind, iters)
        b.record()
        torch.cuda.synchronize()
        best = max(best, ops / (a.elapsed_time(b) / 1e3))
    return best


def test_probe_rates_are_pipe_rates(cuda_lib):
    import torch
    sw = cuda_lib
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    ceiling32 = sms * 128 * 2.07e9               # lanes x the maximum SM clock of this part
    f32_fma = _rate(sw, sw.SWEPT_PROBE_F32_FMA, 20000)
    f32_add = _rate(sw, sw.SWEPT_PROBE_F32_ADD, 20000)
    f64_fma = _rate(sw, sw.SWEPT_PROBE_F64_FMA, 500)
    for r in (f32_fma, f32_add):
        assert 0.5 * ceiling32 < r < 1.02 * ceiling32, (r, ceiling32)
    assert 0 < f64_fma < 0.5 * f32_fma


def test_probe_rejects_bad_arguments(cuda_lib):
    sw = cuda_lib
    for kind, iters in ((7, 10), (sw.SWEPT_PROBE_F32_FMA, 0), (sw.SWEPT_PROBE_F32_FMA, -5)):
        with pytest.raises(sw.SweptError) as ei:
            sw.swept_probe_alu(kind, iters)
        assert ei.value.code == sw.SWEPT_EINVAL
