"""Benchmark of the swept-rule hot path on one GB300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload heat|ks|batch|adjoint|latency|ks_rk2|euler]

Headline workload: 1D heat, periodic, N = 2^24 points, r = 1/4, 20000
sub-timesteps per step, compensated FP32 state, tile B = 1024 (the fastest of
the tile sweep B in {64, ..., 1024}, which is reported too); u0 = uniform[-1,1]
noise plus 16 low modes.  One "step" is one swept_advance of the whole field
through all 20000 sub-timesteps: 41 stages in 4 kernel launches (the first
triangle, one streamed launch for the 38 full diamonds, the last fill, the
remainder stage).

Metric: cell-updates/s = N * nsteps / time.  Every step starts from the same
device-resident input (restored outside the timed events); L2 is flushed
between steps (a 256 MiB write), also outside the timed events.

Printed as one JSON line: the device-timed value, the end-to-end value
through the public API with host buffers, the roofline of the dominant
kernel (its duration from CUDA events the library records around it in
every timed step), the CPU oracle baseline and the SM clocks seen during the
run.  On one GPU the line also carries:
  * peaks     -- the measured FP32 and FP64 arithmetic rates (swept_probe_alu),
                 each with the median SM clock sampled while it ran: the
                 denominators of every roofline fraction below;
  * reports   -- the other workloads, each with its error against the oracle
                 (or a closed form), its dominant kernel's time and its
                 fraction of the measured peak:
                   heat_c1_f64  the headline field in FP64, swept and naive;
                   latency_c0   heat, N = 1024, 2000 steps, FP64 (the latency
                                regime of Sections 4 and 6);
                   ks_c2        Kuramoto-Sivashinsky, N = 2^22, 50000 steps;
                   batch_c3     4096 ragged problems in one persistent launch;
                   adjoint_c4   the KS gradient, N = 2^20, 20000 steps, with 32
                                finite-difference directions;
                   ks_rk2_f1    KS by the two-stage Runge-Kutta rule (Section 6's
                                initial condition), N = 2^22;
                   euler_f2     the Euler equations (Section 7), N = 2^23 and the
                                4096-cell latency regime;
                   uneven_f4    heat on N = 2^24 + 224 (uneven tiles) against
                                N = 2^24, compensated FP32, B = 512.
Algorithmic counts follow the hot-path scope's figures: compensated FP32
heat 11 and KS 22 operations per cell-update against the measured FP32
instruction rate (an add, mul or fma is one operation); FP64 heat 5 and KS 16
FLOP per cell-update against twice the measured FP64 fma rate (an fma is two
FLOP).  The counts the kernels actually execute are given beside them.

--impl reference times the CPU oracle (the plain per-step definition, in
C with OpenMP on the host cores) on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank runs its own replica (the single-problem
path has no cross-GPU exchange); the max time over ranks is reported; the
peaks and reports are measured on one GPU only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

N_POINTS = 1 << 24
NSTEPS = 20000
TILE_B = 1024
HEAT_R = 0.25
METRIC = "cell-updates/s (N x steps / s), swept vs naive stepper, 1 GB300, at stated error"
UNIT = "cell-updates/s"
# Algorithmic work per cell-update (the hot-path scope's figures) and what the kernels execute.
ALGO_OPS_F32C = {"heat": 11, "ks": 22}        # FP32 operations (add/sub/mul/fma = 1)
ALGO_FLOP_F64 = {"heat": 5, "ks": 16}         # FP64 FLOP (fma = 2)
EXEC_OPS_F32C = {"heat": 9, "ks": 16}         # instructions of the compensated cores per update
EXEC_OPS_F64 = {"heat": 3, "ks": 9}
NOMINAL_SMS, NOMINAL_FP32_LANES = 152, 128
# Sources that define the headline kernel (swept_stream_kernel<heat, F32C, 32>): the DRAM
# traffic of a committed ncu summary is used only while their digest matches the one the
# summary records.
HEADLINE_SOURCES = ("swept_ring.cuh", "swept_stage.cuh", "swept_device.cuh", "swept_sync.cuh",
                    "swept_internal.h", "stage_heat_f32c.cu")
HEADLINE_PROFILE = os.path.join(ROOT, "profiles", "swept_stream_kernel_heat_f32c_K32_N2p24.md")
KS_SOURCES = ("swept_ring.cuh", "swept_stage.cuh", "swept_device.cuh", "swept_sync.cuh", "swept_internal.h",
              "stage_ks_f32c.cu")
KS_PROFILE = os.path.join(ROOT, "profiles", "swept_stream_kernel_ks_f32c_K32_N2p22.md")


def workload_config(n_gpus: int):
    return {"workload": "heat1d_periodic_N16777216_r0.25_20000steps_f32c_B1024",
            "N": N_POINTS, "nsteps": NSTEPS, "B": TILE_B, "stencil": "heat 3-point forward Euler",
            "state": "f32 compensated (hi, lo)", "l2": "flushed between steps (256 MiB write)",
            "input": "device-resident, restored between steps", "parallelism": f"replicas x{n_gpus}"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        return parse_clock_lines(lines)


def parse_clock_lines(lines):
    """Median SM clock, max clock and the throttle reasons seen in nvidia-smi CSV lines."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for name, val in zip(names, f[5:9]):
            if val.lower() == "active":
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
            "reasons": sorted(reasons)}


def measured_peaks_file() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def measured_hbm_gbs() -> float:
    """Measured copy bandwidth of this GPU pool (GB/s); 6800 (the fallback) when the file is absent."""
    return float(measured_peaks_file().get("hbm_gbs", 6800.0))


# ------------------------------------------------- committed ncu figures
def code_tokens(text: str) -> str:
    """C++ source without its comments and with every run of whitespace made one space, so
    that the digest of a file changes with its code only (string literals kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':                                  # string literal: copy to its closing quote
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_digest(names=HEADLINE_SOURCES) -> str:
    """sha256 (16 hex digits) of the named kernel sources' code (comments and layout ignored)."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1504_01380_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(code_tokens(f.read()).encode())
    return h.hexdigest()[:16]


def profile_traffic(path: str = HEADLINE_PROFILE, names=HEADLINE_SOURCES):
    """DRAM bytes (read + write) per launch from a committed ncu summary, or None when the
    summary is missing, carries no digest, or was taken from other kernel sources."""
    try:
        text = open(path).read()
    except OSError:
        return None, "no committed capture"
    m = re.search(r"source digest:\s*`?([0-9a-f]{16})", text)
    if not m:
        return None, "capture records no source digest"
    if m.group(1) != source_digest(names):
        return None, "kernel sources changed since the capture"
    rd = re.search(r"dram__bytes_read\.sum\s*=\s*([0-9.]+)\s*Gbyte", text)
    wr = re.search(r"dram__bytes_write\.sum\s*=\s*([0-9.]+)\s*Gbyte", text)
    if not rd or not wr:
        return None, "capture has no DRAM byte counts"
    return (float(rd.group(1)) + float(wr.group(1))) * 1e9, "ncu capture of the current sources"


# ---------------------------------------------------------- GPU timing
def cuda_time(fn, stream=None):
    """Seconds of fn() on the device: CUDA events on the current stream, synchronised."""
    import torch
    s = stream or torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def measure_alu_peaks(dev_index: int) -> dict:
    """FP32 and FP64 operation rates of this GPU (swept_probe_alu: dependency-free chains over
    every SM), each the best of five launches of about 100 ms, with the SM clocks sampled while
    that probe ran."""
    import torch
    import paper_1504_01380_gb300 as sw
    out = {}
    kinds = (("f32_fma", sw.SWEPT_PROBE_F32_FMA), ("f32_add", sw.SWEPT_PROBE_F32_ADD),
             ("f64_fma", sw.SWEPT_PROBE_F64_FMA), ("f64_add", sw.SWEPT_PROBE_F64_ADD))
    for name, kind in kinds:
        it = 64
        ops = 0.0
        while True:                                  # size one launch to about 100 ms
            t = cuda_time(lambda: sw.swept_probe_alu(kind, it))
            if t > 0.02 or it > (1 << 34):
                break
            it *= 4
        it = max(1, int(it * 0.1 / max(t, 1e-6)))
        with ClockSampler(dev_index) as clk:
            best = 0.0
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ops = sw.swept_probe_alu(kind, it)
                b.record()
                torch.cuda.synchronize()
                best = max(best, ops / (a.elapsed_time(b) / 1e3))
        c = clk.summary()
        out[name] = {"ops_per_s": best, "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")}
    out["fp32_ops_per_s"] = max(out["f32_fma"]["ops_per_s"], out["f32_add"]["ops_per_s"])
    out["fp64_flop_per_s"] = 2.0 * out["f64_fma"]["ops_per_s"]
    out["how"] = ("swept_probe_alu: 8 independent add or fma chains per thread, every SM at full "
                  "residency; best of 5 launches of ~100 ms; an add or fma is one operation, FP64 "
                  "FLOP/s = 2 x the fma rate")
    return out


def peak_block(peaks, kind: str):
    """(peak, unit, source) for the roofline: 'fp32' operations/s or 'fp64' FLOP/s, measured."""
    sm_max = float(measured_peaks_file().get("sm_max_mhz", 2070.0))
    if kind == "fp32":
        nominal = NOMINAL_SMS * NOMINAL_FP32_LANES * sm_max * 1e6
        if peaks:
            p = peaks["fp32_ops_per_s"]
            clk = peaks["f32_fma"]["sm_mhz"]
            return p, "FP32 ops/s", f"measured: swept_probe_alu FP32 chains at {clk} MHz", nominal
        return nominal, "FP32 ops/s", f"nominal: 152 SMs x 128 lanes x {sm_max:.0f} MHz", nominal
    if peaks:
        clk = peaks["f64_fma"]["sm_mhz"]
        return peaks["fp64_flop_per_s"], "FP64 FLOP/s", f"measured: swept_probe_alu FP64 fma chains x 2 at {clk} MHz", None
    return None, "FP64 FLOP/s", "not measured", None


def roofline(work_per_s: float, peak, unit: str, source: str, **extra):
    d = {"bound": "alu", "achieved": work_per_s / 1e12, "peak": (peak / 1e12) if peak else None,
         "unit": "T" + unit, "frac": (work_per_s / peak) if peak else None, "peak_source": source}
    d.update(extra)
    return d


# ------------------------------------------------------------ CPU oracle
def time_oracle(target_s: float = 15.0):
    """The oracle (compensated FP32 per-step stepping, OpenMP) on a bounded sample of the
    headline field; also returns the sample's result and step count, which the GPU path must
    reproduce bit for bit."""
    import oracle
    u0 = workloads.heat_noise_modes(N_POINTS)
    hi, lo = oracle.split_f32c(u0)
    threads = cores_used()
    oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi, lo, 2, threads)      # thread start-up
    t0 = time.perf_counter()
    oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi, lo, 8, threads)
    dt = max(time.perf_counter() - t0, 1e-6) / 8
    steps = max(2, min(NSTEPS, int(target_s / dt)))
    t0 = time.perf_counter()
    out = oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi, lo, steps, threads)
    el = time.perf_counter() - t0
    # the same oracle on one core, a shorter sample
    steps1 = max(1, min(steps, int(2.0 / (dt * threads))))
    t0 = time.perf_counter()
    oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi, lo, steps1, 1)
    el1 = time.perf_counter() - t0
    return ({"value": N_POINTS * steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
             "sample": f"N=2^24, first {steps} of 20000 sub-timesteps, {el:.1f} s",
             "one_core": {"value": N_POINTS * steps1 / el1, "sample": f"N=2^24, {steps1} sub-timesteps"}},
            steps, out)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    u0 = workloads.heat_noise_modes(N_POINTS)
    hi0, lo0 = oracle.split_f32c(u0)
    threads = cores_used()
    # size one step so that warmup + steps take about two minutes in total
    t0 = time.perf_counter()
    oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi0, lo0, 2, threads)
    per = max(time.perf_counter() - t0, 1e-6) / 2
    budget = 120.0 / max(1, args.steps + args.warmup)
    sample_steps = max(1, min(NSTEPS, int(budget / per)))
    for _ in range(args.warmup):
        oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi0, lo0, sample_steps, threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.advance_f32c(oracle.HEAT, [HEAT_R], hi0, lo0, sample_steps, threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = N_POINTS * sample_steps * args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32c", "data": "synthetic",
            "impl": "reference", "config": workload_config(args.gpus),
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value, "unit": UNIT,
                             "sample": f"N=2^24, {sample_steps} of 20000 sub-timesteps per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def exact_heat(u0: np.ndarray, r: float, nsteps: int) -> np.ndarray:
    """Closed form of periodic forward-Euler heat stepping: Fourier mode k is multiplied by
    g_k = 1 - 4 r sin^2(pi k / N) per step."""
    n = u0.size
    k = np.arange(n // 2 + 1)
    g = 1.0 - 4.0 * r * np.sin(np.pi * k / n) ** 2
    return np.fft.irfft(np.fft.rfft(u0) * g ** nsteps, n)


# ------------------------------------------------------------------ GPU
def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_1504_01380_gb300 as sw
    sw.load()

    # measured arithmetic peaks (one GPU runs): the roofline denominators
    peaks = measure_alu_peaks(dev.index) if world == 1 else None

    u0 = workloads.heat_noise_modes(N_POINTS)
    u0_dev = torch.tensor(u0, device=dev)
    plan = sw.swept_plan(N_POINTS, 1, sw.SWEPT_HEAT, [HEAT_R], sw.SWEPT_F32C, TILE_B)
    pristine = sw.swept_f32c_split(u0_dev)
    u = torch.empty_like(pristine)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    h = plan.h
    # events around the ring launch of every advance: the dominant kernel's own duration
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIME_RING, 1)
    ring_ms, launches = [], []

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def one(timed_list=None):
        u.copy_(pristine)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sw.swept_advance(plan, u, NSTEPS)
        e1.record(stream)
        if timed_list is not None:
            timed_list.append((e0, e1))
            n_all, n_ring, t_ring = sw.swept_plan_last_advance(plan)    # waits for the ring launch
            launches.append((n_all, n_ring))
            ring_ms.append(t_ring)

    for _ in range(args.warmup):
        one()
    barrier()
    events = []
    with ClockSampler(dev.index) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            one(events)
        barrier()
        wall = time.perf_counter() - wall0
    ms = [a.elapsed_time(b) for a, b in events]
    t_dev = sum(ms) / 1e3
    if world > 1:
        tt = torch.tensor([t_dev], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_dev = float(tt.item())
    updates = N_POINTS * NSTEPS * args.steps * world
    value = updates / t_dev
    clocks = clk.summary()

    # ---- end to end through the public API: pinned host in, pinned host out
    host_in = torch.tensor(u0).pin_memory()
    host_out = torch.empty(N_POINTS, dtype=torch.float64).pin_memory()
    dev64 = torch.empty(N_POINTS, dtype=torch.float64, device=dev)

    def e2e_step():
        dev64.copy_(host_in, non_blocking=True)
        sw.swept_f32c_split(dev64, out=u)
        sw.swept_advance(plan, u, NSTEPS)
        sw.swept_f32c_merge(u, out=dev64)
        host_out.copy_(dev64, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1)
        e2e_times.append(cuda_time(e2e_step, stream))
    e2e_value = N_POINTS * NSTEPS * world / statistics.mean(e2e_times)

    # stated error: compensated result against the exact Fourier solution
    got = host_out.numpy()
    exact = exact_heat(u0, HEAT_R, NSTEPS)
    scale = float(np.max(np.abs(u0)))
    max_err = float(np.max(np.abs(got - exact)) / scale)

    # ---- comparison runs (one step each, outside the timed region)
    def timed(fn, dst, src):
        dst.copy_(src)
        flush.fill_(1)
        return cuda_time(fn, stream)

    naive_f32c = N_POINTS * NSTEPS / timed(lambda: sw.swept_naive_advance(plan, u, NSTEPS), u, pristine)

    # plain binary32 state (diagnostic precision): rate and error against the exact solution
    plan32 = sw.swept_plan(N_POINTS, 1, sw.SWEPT_HEAT, [HEAT_R], sw.SWEPT_F32, TILE_B)
    u32p = u0_dev.float()
    swept_f32 = N_POINTS * NSTEPS / timed(lambda: sw.swept_advance(plan32, u32p, NSTEPS), u32p, u0_dev.float())
    err_f32 = float(np.max(np.abs(u32p.double().cpu().numpy() - exact)) / scale)
    plan32.destroy()
    del u32p

    # tile sweep B in {64, ..., 1024} (compensated FP32, one step each)
    sweep = {}
    for tb in (64, 128, 256, 512, 1024):
        pb = sw.swept_plan(N_POINTS, 1, sw.SWEPT_HEAT, [HEAT_R], sw.SWEPT_F32C, tb)
        sweep[str(tb)] = N_POINTS * NSTEPS / timed(lambda: sw.swept_advance(pb, u, NSTEPS), u, pristine)
        pb.destroy()

    # FP64 reductions of the compensated state (sum, half sum of squares; dot with an FP64
    # vector): bytes read over time, L2 flushed before each
    red = {}
    for name, what, nbytes in (("sum", sw.SWEPT_SUM, 8 * N_POINTS), ("half_sumsq", sw.SWEPT_HALF_SUMSQ, 8 * N_POINTS),
                               ("dot", sw.SWEPT_DOT, 16 * N_POINTS)):
        ts = []
        for _ in range(5):
            flush.fill_(1)
            ts.append(cuda_time(lambda: sw.swept_reduce(plan, u, what, v=u0_dev if what == sw.SWEPT_DOT else None),
                                stream))
        red[name] = {"bytes": nbytes, "ms": statistics.median(ts) * 1e3,
                     "GB/s": nbytes / statistics.median(ts) / 1e9}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    hbm = measured_hbm_gbs()
    # Dominant kernel: the streamed ring kernel (heat, compensated FP32, K = 32), one
    # launch per step running the q - 1 = 38 full-diamond stages (N x h updates each);
    # the other three launches are the first triangle, the last fill and the remainder.
    # Its duration comes from the library's events around it in every timed step.
    n_all, n_ring = launches[0]
    q = NSTEPS // h
    ring_updates = N_POINTS * h * (q - 1) / n_ring
    avg_launch_s = statistics.mean(ring_ms) / 1e3 / n_ring
    peak, unit, source, nominal = peak_block(peaks, "fp32")
    traffic, traffic_note = profile_traffic()
    roof = roofline(ALGO_OPS_F32C["heat"] * ring_updates / avg_launch_s, peak, unit, source,
                    kernel="swept_stream_kernel<heat,f32c,K=32>",
                    traffic=traffic, traffic_unit="DRAM bytes per launch (ncu)", traffic_note=traffic_note,
                    algorithmic_edge_bytes_per_launch=2 * 16 * N_POINTS * (q - 1) / n_ring,
                    ops_per_update=ALGO_OPS_F32C["heat"], executed_ops_per_update=EXEC_OPS_F32C["heat"],
                    per_launch_ops=ALGO_OPS_F32C["heat"] * ring_updates, avg_launch_ms=avg_launch_s * 1e3,
                    launches_per_step=n_all, ring_launches_per_step=n_ring,
                    frac_whole_advance=ALGO_OPS_F32C["heat"] * value / world / peak if peak else None,
                    frac_executed=EXEC_OPS_F32C["heat"] * ring_updates / avg_launch_s / peak if peak else None,
                    frac_of_nominal=ALGO_OPS_F32C["heat"] * ring_updates / avg_launch_s / nominal)
    cpu, bitexact = None, None
    reports = None
    if world == 1:
        cpu, steps_s, (ohi, olo) = time_oracle()
        # the GPU path on the oracle's sample: bit for bit
        u.copy_(pristine)
        sw.swept_advance(plan, u, steps_s)
        gh = u.cpu().numpy()
        bitexact = bool(np.array_equal(gh[:N_POINTS], ohi) and np.array_equal(gh[N_POINTS:], olo))
        cpu["gpu_bit_exact_on_sample"] = bitexact
        plan.destroy()
        del u, pristine, host_in, host_out, dev64
        torch.cuda.empty_cache()
        if args.reports == "all":
            reports = run_reports(peaks, dev, flush)
    naive_roof = hbm * 1e9 / 16.0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
            "ms_per_step_median": statistics.median(ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32c",
            "data": "synthetic", "config": workload_config(world),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N_POINTS,
                    "d2h_bytes_per_step": 8 * N_POINTS},
            "gpu_launches": sum(n for n, _ in launches),
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "max_err_vs_exact": max_err,
            "compare": {"naive_f32c": naive_f32c, "swept_f32_plain": swept_f32,
                        "max_err_f32_plain_vs_exact": err_f32,
                        "naive_hbm_roof_16B": naive_roof, "swept_over_naive_hbm_roof": value / world / naive_roof,
                        "swept_over_naive_f32c": value / world / naive_f32c,
                        "tile_sweep_f32c": sweep,
                        "reductions_f64": {k: dict(v, frac_of_measured_hbm=v["GB/s"] / hbm)
                                           for k, v in red.items()}},
            "peaks": peaks, "reports": reports,
            "wall_s": wall}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- reports
def run_reports(peaks, dev, flush) -> dict:
    """Every other workload of the benchmark suite on this GPU, each with its error, its
    dominant kernel's time and its fraction of the measured peak (one GPU runs only)."""
    import torch
    out = {}
    for name, fn in (("heat_c1_f64", report_heat_f64), ("latency_c0", report_latency_c0),
                     ("ks_c2", report_ks_c2), ("batch_c3", report_batch_c3),
                     ("adjoint_c4", report_adjoint_c4), ("ks_rk2_f1", report_ks_rk2_f1),
                     ("euler_f2", report_euler_f2), ("uneven_f4", report_uneven_f4)):
        t0 = time.perf_counter()
        try:
            out[name] = fn(peaks, flush)
        except Exception as e:        # one report's failure must not hide the others
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


def report_heat_f64(peaks, flush):
    """The headline field (heat, N = 2^24, 20000 steps) in FP64: swept (streamed ring) and naive."""
    import torch
    import paper_1504_01380_gb300 as sw
    u0 = workloads.heat_noise_modes(N_POINTS)
    u0_dev = torch.tensor(u0, device="cuda")
    u = u0_dev.clone()
    plan = sw.swept_plan(N_POINTS, 1, sw.SWEPT_HEAT, [HEAT_R], sw.SWEPT_F64, TILE_B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIME_RING, 1)

    def run(fn):
        u.copy_(u0_dev)
        flush.fill_(1)
        return cuda_time(fn)

    run(lambda: sw.swept_advance(plan, u, 2 * plan.h + 1))            # warm-up
    t_sw = run(lambda: sw.swept_advance(plan, u, NSTEPS))
    n_all, n_ring, ring_ms = sw.swept_plan_last_advance(plan)
    err = float(np.max(np.abs(u.cpu().numpy() - exact_heat(u0, HEAT_R, NSTEPS))) / np.max(np.abs(u0)))
    t_nv = run(lambda: sw.swept_naive_advance(plan, u, NSTEPS))
    h = plan.h
    q = NSTEPS // h
    plan.destroy()
    peak, unit, source, _ = peak_block(peaks, "fp64")
    ring_updates = N_POINTS * h * (q - 1)
    rate_ring = ring_updates / (ring_ms / 1e3) if ring_ms > 0 else None
    work = ALGO_FLOP_F64["heat"]
    return {"workload": "heat1d_periodic_N16777216_r0.25_20000steps_f64_B1024", "unit": UNIT,
            "swept": N_POINTS * NSTEPS / t_sw, "naive": N_POINTS * NSTEPS / t_nv,
            "swept_over_naive": t_nv / t_sw, "max_err_vs_exact": err,
            "error_reference": "exact Fourier solution (mode k scaled by g_k per step), relative to max|u0|",
            "launches": n_all,
            "roofline": roofline(work * rate_ring if rate_ring else 0.0, peak, unit, source,
                                 kernel="swept_stream_kernel<heat,f64,K=32>", avg_launch_ms=ring_ms / max(1, n_ring),
                                 flop_per_update=work, executed_ops_per_update=EXEC_OPS_F64["heat"],
                                 naive_frac=work * N_POINTS * NSTEPS / t_nv / peak if peak else None)}


def report_uneven_f4(peaks, flush):
    """Arbitrary N: the headline scheme (heat, compensated FP32, B = 512, 5000 steps) on
    N = 2^24 + 224 (seven wide windows of 544 points) against the even N = 2^24, both with their
    diamonds in one streamed launch; the uneven result against the naive stepper bit for bit."""
    import torch
    import paper_1504_01380_gb300 as sw
    nsteps, B = 5000, 512
    out = {}
    for name, n in (("even", N_POINTS), ("uneven", N_POINTS + 224)):
        u0 = sw.swept_f32c_split(torch.tensor(workloads.uniform(n, 5), device="cuda"))
        u = u0.clone()
        plan = sw.swept_plan(n, 1, sw.SWEPT_HEAT, [HEAT_R], sw.SWEPT_F32C, B)

        def run(fn):
            u.copy_(u0)
            flush.fill_(1)
            return cuda_time(fn)

        run(lambda: sw.swept_advance(plan, u, 2 * plan.h + 1))            # warm-up
        t = min(run(lambda: sw.swept_advance(plan, u, nsteps)) for _ in range(3))
        launches = sw.swept_plan_last_advance(plan)[:2]
        rec = {"N": n, "swept": n * nsteps / t, "launches": launches[0], "ring_launches": launches[1]}
        if name == "uneven":
            got = u.clone()
            u.copy_(u0)
            sw.swept_naive_advance(plan, u, nsteps)
            rec["bit_exact_vs_naive"] = bool(torch.equal(got, u))
            rec["wide_windows"] = -(-(n % B) // 32)                 # ceil((N mod B) / 32r), r = 1
        plan.destroy()
        out[name] = rec
    return {"workload": "heat1d_N16777440_r0.25_5000steps_f32c_B512", "unit": UNIT,
            "even": out["even"], "uneven": out["uneven"],
            "uneven_over_even": out["uneven"]["swept"] / out["even"]["swept"]}


def report_latency_c0(peaks, flush):
    """Heat, N = 1024, r = 1/4, 2000 steps, FP64, B = 32: the latency regime.  Per sub-timestep:
    the swept advance in one thread block cluster (the stage edges in shared memory, a cluster
    barrier between stages: the default where the problem fits one cluster) and with one launch
    per stage (graph-replayed), against the naive stepper with its steps in one cluster (one
    cluster barrier per step) and with one launch per step (graph-replayed); Eq. 1 fitted over
    B for both kinds of stage boundary; the compensated FP32 state."""
    import torch
    import paper_1504_01380_gb300 as sw
    from paper_1504_01380_gb300 import tune
    n, nsteps = 1024, 2000
    u0 = workloads.heat_modes(n, 8)
    u0_dev = torch.tensor(u0, device="cuda")
    u = u0_dev.clone()

    def per_sub(fn, x, x0, reps=5):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            x.copy_(x0)
            best = min(best, cuda_time(fn))
        return best / nsteps

    def swept_times(dtype, x, x0, widths):
        res, launch = {}, {}
        for B in widths:
            plan = sw.swept_plan(n, 1, sw.SWEPT_HEAT, [HEAT_R], dtype, B)
            t = per_sub(lambda: sw.swept_advance(plan, x, nsteps), x, x0)
            if sw.swept_plan_last_advance(plan)[0] == 1:        # one cluster launch (K <= 4)
                res[B] = t
            sw.swept_plan_set(plan, sw.SWEPT_OPT_RESIDENT, 0)
            sw.swept_plan_set(plan, sw.SWEPT_OPT_GRAPH, 1)
            launch[B] = per_sub(lambda: sw.swept_advance(plan, x, nsteps), x, x0)
            plan.destroy()
        return res, launch

    def naive_times(dtype, x, x0):
        plan = sw.swept_plan(n, 1, sw.SWEPT_HEAT, [HEAT_R], dtype, 32)
        g = torch.cuda.CUDAGraph()
        x.copy_(x0)
        with torch.cuda.graph(g):
            sw.swept_naive_advance(plan, x, nsteps)
        t_graph = per_sub(g.replay, x, x0, reps=3)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_NAIVE_RESIDENT, 1)
        t_res = per_sub(lambda: sw.swept_naive_advance(plan, x, nsteps), x, x0)
        plan.destroy()
        return t_graph, t_res

    widths = (32, 64, 128, 256)
    res, launch = swept_times(sw.SWEPT_F64, u, u0_dev, widths)
    naive, naive_res = naive_times(sw.SWEPT_F64, u, u0_dev)
    # the result of each path at B = 32
    got = {}
    for resident in (1, 0):
        plan = sw.swept_plan(n, 1, sw.SWEPT_HEAT, [HEAT_R], sw.SWEPT_F64, 32)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_RESIDENT, resident)
        u.copy_(u0_dev)
        sw.swept_advance(plan, u, nsteps)
        got[resident] = u.cpu().numpy()
        if resident == 0:
            launches, h32 = sw.swept_plan_last_advance(plan)[0], plan.h
        plan.destroy()
    # compensated FP32 state
    c0 = sw.swept_f32c_split(u0_dev)
    c = c0.clone()
    res32, launch32 = swept_times(sw.SWEPT_F32C, c, c0, (32, 64))
    naive32, naive32_res = naive_times(sw.SWEPT_F32C, c, c0)
    fit = tune.fit_eq1([(B, t) for B, t in launch.items()])
    fit_res = tune.fit_eq1([(B, t) for B, t in res.items()])
    exact = exact_heat(u0, HEAT_R, nsteps)
    err = float(np.max(np.abs(got[1] - exact)) / np.max(np.abs(u0)))
    oracle_leg = cpu_leg_latency(u0, nsteps, got[1])
    oracle_leg["stage_launches_equal_resident"] = bool(np.array_equal(got[0], got[1]))
    t32, tl32 = res[32], launch[32]
    ns = lambda d: {str(B): t * 1e9 for B, t in d.items()}
    eq1 = lambda f: {"s_ns": f["s"] * 1e9, "tau_ns": f["tau"] * 1e9, "n_star": f["n_star"]} if f else None
    return {"workload": "heat1d_N1024_r0.25_2000steps_f64_B32", "unit": "ns per sub-timestep",
            "swept_ns": t32 * 1e9, "swept_path": "one thread block cluster (stage edges in shared memory, cluster barriers)",
            "swept_ns_by_B": ns(res),
            "swept_stage_launches_graph_ns": tl32 * 1e9, "swept_stage_launches_graph_ns_by_B": ns(launch),
            "stage_launches": launches,
            "naive_resident_ns": naive_res * 1e9, "naive_graph_ns": naive * 1e9,
            "speedup_vs_naive_resident": naive_res / t32, "speedup_vs_naive_graph": naive / t32,
            "stage_launches_speedup_vs_naive_graph": naive / tl32,
            "max_err_vs_closed_form": err,
            "error_reference": "closed form sum_k g_k^n (a_k sin + b_k cos), relative to max|u0|",
            "f32c": {"swept_ns_by_B": ns(res32), "swept_stage_launches_graph_ns_by_B": ns(launch32),
                     "naive_resident_ns": naive32_res * 1e9, "naive_graph_ns": naive32 * 1e9,
                     "speedup_vs_naive_resident": naive32_res / min(res32.values()),
                     "speedup_vs_naive_graph": naive32 / min(res32.values())},
            "eq1_fit_stage_launches": eq1(fit), "eq1_fit_resident": eq1(fit_res),
            "roofline": {"bound": "latency", "achieved": tl32 * 1e9, "unit": "ns per sub-timestep",
                         "peak": naive * 1e9 / h32, "frac": (naive / h32) / tl32,
                         "kernel": "per-stage launches (graph-replayed)",
                         "peak_source": ("measured: one kernel boundary (the graph-replayed naive stepper's "
                                         "time per sub-timestep) paid once per stage of h = 16 sub-timesteps; "
                                         "the rest of the time is the per-level dependence chain of one warp")},
            "cpu_baseline": oracle_leg}



def cpu_leg_latency(u0, nsteps, got):
    """Oracle leg of the latency report: the oracle on the same 1024-point run, timed on the host
    cores, and the GPU result compared with it bit for bit."""
    import oracle
    t0 = time.perf_counter()
    want = oracle.advance_f64(oracle.HEAT, [HEAT_R], u0, nsteps, 1)
    el = time.perf_counter() - t0
    return {"kind": "oracle", "cores": 1, "value": u0.size * nsteps / el, "unit": UNIT,
            "sample": f"the whole workload, N=1024 x {nsteps} sub-timesteps, one thread",
            "gpu_bit_exact": bool(np.array_equal(got, want))}


def report_ks_c2(peaks, flush):
    """KS (forward Euler), N = 2^22, dx = 0.5, dt = 0.002, 50000 steps, u0 = 0.1 smooth^10(N(0,1)).

    Compensated FP32 (B = 1024, streamed ring; B = 512 beside it) over the full 50000 steps
    against the naive stepper; FP64 swept (B = 1024) and naive over 5000 steps (both
    FP64-pipe-bound).  Error: the
    compensated state after 2000 steps against the FP64 oracle (after 50000 steps the chaotic
    dynamics have amplified rounding differences to the size of the solution); the FP64 GPU
    state after 2000 steps must equal the oracle's bit for bit.
    """
    import torch
    import paper_1504_01380_gb300 as sw
    n, nsteps, nshort, nerr, B = 1 << 22, 50000, 5000, 2000, 1024
    prm = [workloads.KS_DT, workloads.KS_DX]
    u0 = workloads.ks_smoothed(n)
    u64 = torch.tensor(u0, device="cuda")
    u32 = sw.swept_f32c_split(u64)
    u = u32.clone()

    def run(fn, dst, src):
        dst.copy_(src)
        flush.fill_(1)
        return cuda_time(fn)

    sweep = {}
    p512 = sw.swept_plan(n, 2, sw.SWEPT_KS, prm, sw.SWEPT_F32C, 512)
    run(lambda: sw.swept_advance(p512, u, nerr), u, u32)
    sweep["512"] = n * nsteps / run(lambda: sw.swept_advance(p512, u, nsteps), u, u32)
    p512.destroy()
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, prm, sw.SWEPT_F32C, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIME_RING, 1)
    run(lambda: sw.swept_advance(plan, u, nerr), u, u32)                      # warm-up
    f32_2000 = sw.swept_f32c_merge(u).cpu().numpy()
    t = run(lambda: sw.swept_advance(plan, u, nsteps), u, u32)
    n_all, n_ring, ring_ms = sw.swept_plan_last_advance(plan)
    h = plan.h
    t_nv = run(lambda: sw.swept_naive_advance(plan, u, nshort), u, u32)
    plan.destroy()
    v = u64.clone()
    p64 = sw.swept_plan(n, 2, sw.SWEPT_KS, prm, sw.SWEPT_F64, B)
    t64 = run(lambda: sw.swept_advance(p64, v, nshort), v, u64)
    t64n = run(lambda: sw.swept_naive_advance(p64, v, nshort), v, u64)
    run(lambda: sw.swept_advance(p64, v, nerr), v, u64)
    f64_2000 = v.cpu().numpy()
    p64.destroy()
    leg, want = cpu_leg_ks(u0, prm, nerr)
    scale = float(np.max(np.abs(want)))
    q = nsteps // h
    ring_updates = n * h * (q - 1)
    peak, unit, source, _ = peak_block(peaks, "fp32")
    leg["gpu_f64_bit_exact"] = bool(np.array_equal(f64_2000, want))
    rate = n * nsteps / t
    traffic, traffic_note = profile_traffic(KS_PROFILE, KS_SOURCES)
    sweep[str(B)] = rate
    return {"workload": f"ks1d_N{n}_dx0.5_dt0.002_{nsteps}steps_f32c_B{B}", "unit": UNIT, "tile_sweep": sweep,
            "swept": rate, "naive": n * nshort / t_nv, "swept_over_naive": rate / (n * nshort / t_nv),
            "naive_hbm_roof_16B": measured_hbm_gbs() * 1e9 / 16,
            "f64": {"swept": n * nshort / t64, "naive": n * nshort / t64n, "steps": nshort},
            "max_err_f32c_vs_oracle_f64_after_2000": float(np.max(np.abs(f32_2000 - want))) / scale,
            "error_reference": "FP64 oracle after 2000 steps, relative to its max|u|; bar 1e-5",
            "launches": n_all,
            "roofline": roofline(ALGO_OPS_F32C["ks"] * ring_updates / (ring_ms / 1e3), peak, unit, source,
                                 kernel="swept_stream_kernel<ks,f32c,K=32>", avg_launch_ms=ring_ms / max(1, n_ring),
                                 traffic=traffic, traffic_unit="DRAM bytes per launch (ncu)",
                                 traffic_note=traffic_note,
                                 algorithmic_edge_bytes_per_launch=2 * 16 * n * (q - 1),
                                 ops_per_update=ALGO_OPS_F32C["ks"], executed_ops_per_update=EXEC_OPS_F32C["ks"],
                                 frac_executed=EXEC_OPS_F32C["ks"] * ring_updates / (ring_ms / 1e3) / peak
                                 if peak else None,
                                 frac_whole_advance=ALGO_OPS_F32C["ks"] * rate / peak if peak else None),
            "cpu_baseline": leg}


def cpu_leg_ks(u0, prm, nsteps):
    """Oracle leg of the KS report: the FP64 oracle over the first 2000 steps of the full field on
    the host cores (timed), whose result is the error reference."""
    import oracle
    threads = cores_used()
    t0 = time.perf_counter()
    want = oracle.advance_f64(oracle.KS, prm, u0, nsteps, threads)
    el = time.perf_counter() - t0
    return ({"kind": "oracle", "cores": threads, "value": u0.size * nsteps / el, "unit": UNIT,
             "sample": f"N=2^22, first {nsteps} of 50000 steps, FP64, {el:.1f} s"}, want)


def report_batch_c3(peaks, flush):
    """4096 ragged problems (half heat, half KS), compensated FP32, one persistent launch under a
    CUDA graph, against the naive batched stepper (one launch per time step over every active
    problem) and one naive launch sequence per problem (a seeded sample)."""
    import torch
    import paper_1504_01380_gb300 as sw
    from paper_1504_01380_gb300 import tune
    kinds, lengths, steps = workloads.batch_problems()
    prm = {0: (HEAT_R, 0.0), 1: (workloads.KS_DT, workloads.KS_DX)}
    problems = [(int(k), int(n), int(s), prm[int(k)]) for k, n, s in zip(kinds, lengths, steps)]
    choice = tune.tune_batch(problems, sw.SWEPT_F32C)
    batch = sw.swept_batch_plan(problems, sw.SWEPT_F32C, choice["B_heat"], choice["B_ks"])
    states = workloads.batch_initial(kinds, lengths)
    pool = torch.zeros(batch.pool_bytes, dtype=torch.uint8, device="cuda")
    for off, s0 in zip(batch.offsets, states):
        seg = pool[off:off + 8 * len(s0)].view(torch.float32)
        sw.swept_f32c_split(torch.tensor(s0, device="cuda"), out=seg)
    pristine = pool.clone()
    work = {0: float(np.sum(np.where(kinds == 0, lengths * steps, 0).astype(np.float64))),
            1: float(np.sum(np.where(kinds == 1, lengths * steps, 0).astype(np.float64)))}
    total = work[0] + work[1]

    def run(fn):
        pool.copy_(pristine)
        flush.fill_(1)
        return cuda_time(fn)

    run(lambda: sw.swept_advance_batch(batch, pool))                          # warm-up (graph capture)
    times = [run(lambda: sw.swept_advance_batch(batch, pool)) for _ in range(2)]
    status = sw.swept_batch_status(batch)
    t = min(times)
    result = pool.clone()
    t_nb = run(lambda: sw.swept_batch_naive_advance(batch, pool))             # allocates on first use
    t_nb = run(lambda: sw.swept_batch_naive_advance(batch, pool))
    # one naive launch sequence per problem, a seeded sample of 16
    rng = np.random.default_rng(1)
    sample = rng.choice(len(problems), 16, replace=False)
    nu, ns = 0.0, 0.0
    for i in sample:
        st, n, nst, p = problems[i]
        plan = sw.swept_plan(n, sw.RADIUS[st], st, p[: 1 if st == 0 else 2], sw.SWEPT_F32C, 0)
        uu = sw.swept_f32c_split(torch.tensor(states[i], device="cuda"))
        ns += cuda_time(lambda: sw.swept_naive_advance(plan, uu, nst))
        nu += n * nst
        plan.destroy()
    # oracle leg: a seeded sample of small problems, bit for bit, and the compensated state's error
    leg = cpu_leg_batch(problems, states, batch.offsets, result.cpu().numpy())
    # KS problems over at most 2000 steps (beyond, the chaotic dynamics amplify rounding
    # differences to the size of the solution): a sub-batch of six seeded KS problems
    ks_idx = [i for i, (st, n, _, _) in enumerate(problems) if st == 1 and n <= 16384]
    ks_pick = sorted(np.random.default_rng(8).choice(ks_idx, 6, replace=False).tolist())
    sub = [(1, problems[i][1], min(problems[i][2], 2000), problems[i][3]) for i in ks_pick]
    sb = sw.swept_batch_plan(sub, sw.SWEPT_F32C, choice["B_heat"], choice["B_ks"])
    spool = torch.zeros(sb.pool_bytes, dtype=torch.uint8, device="cuda")
    for off, i in zip(sb.offsets, ks_pick):
        seg = spool[off:off + 8 * len(states[i])].view(torch.float32)
        sw.swept_f32c_split(torch.tensor(states[i], device="cuda"), out=seg)
    sw.swept_advance_batch(sb, spool)
    leg["ks_2000"] = cpu_leg_batch_ks(sub, [states[i] for i in ks_pick], sb.offsets, spool.cpu().numpy())
    sb.destroy()
    info = batch.info()
    batch.destroy()
    peak, unit, source, _ = peak_block(peaks, "fp32")
    ops = ALGO_OPS_F32C["heat"] * work[0] + ALGO_OPS_F32C["ks"] * work[1]
    exe = EXEC_OPS_F32C["heat"] * work[0] + EXEC_OPS_F32C["ks"] * work[1]
    return {"workload": "batch_4096_ragged_heat_ks_f32c", "unit": UNIT, "problems": len(problems),
            "sum_N_x_steps": total, "swept": total / t, "status": status,
            "naive_batched": total / t_nb, "swept_over_naive_batched": t_nb / t,
            "naive_per_problem": {"value": nu / ns, "sample": "16 seeded problems, one launch per sub-timestep"},
            "B_heat": choice["B_heat"], "B_ks": choice["B_ks"], "tuning": choice["rates"], **info,
            "roofline": roofline(ops / t, peak, unit, source, kernel="swept_batch_kernel (one launch)",
                                 avg_launch_ms=t * 1e3, ops_per_update={"heat": 11, "ks": 22},
                                 frac_executed=exe / t / peak if peak else None),
            "cpu_baseline": leg}


def cpu_leg_batch(problems, states, offsets, pool_bytes: np.ndarray, count: int = 12):
    """Oracle leg of the batch report: a seeded sample of problems with at most 2e8 cell-updates,
    each stepped by the compensated oracle (one thread, timed) and compared bit for bit with the
    GPU batch result; the compensated result's error against the FP64 oracle (heat at the final
    step; KS over at most 2000 steps is covered by the KS report)."""
    import oracle
    small = [i for i, (_, n, s, _) in enumerate(problems) if n * s <= 2e8]
    rng = np.random.default_rng(7)
    pick = sorted(rng.choice(small, min(count, len(small)), replace=False).tolist())
    exact, worst, el, upd = True, 0.0, 0.0, 0.0
    for i in pick:
        st, n, nst, p = problems[i]
        prm = list(p[: 1 if st == 0 else 2])
        hi, lo = oracle.split_f32c(states[i])
        t0 = time.perf_counter()
        whi, wlo = oracle.advance_f32c(st, prm, hi, lo, nst, 1)
        el += time.perf_counter() - t0
        upd += n * nst
        seg = pool_bytes[offsets[i]:offsets[i] + 8 * n].view(np.float32)
        exact = exact and np.array_equal(seg[:n], whi) and np.array_equal(seg[n:], wlo)
        if st == 0:
            w64 = oracle.advance_f64(st, prm, states[i], nst, 1)
            got = seg[:n].astype(np.float64) + seg[n:].astype(np.float64)
            worst = max(worst, float(np.max(np.abs(got - w64)) / np.max(np.abs(states[i]))))
    return {"kind": "oracle", "cores": 1, "value": upd / el, "unit": UNIT,
            "sample": f"{len(pick)} seeded problems of at most 2e8 cell-updates, one thread each",
            "gpu_bit_exact": bool(exact), "max_err_heat_f32c_vs_oracle_f64": worst}


def cpu_leg_batch_ks(sub, states, offsets, pool_bytes: np.ndarray):
    """Oracle leg of the batch report's KS sub-batch (at most 2000 steps each): the compensated
    result against the compensated oracle bit for bit and against the FP64 oracle (bar 1e-5
    relative to max|u|)."""
    import oracle
    exact, worst = True, 0.0
    for (st, n, nst, p), u0, off in zip(sub, states, offsets):
        prm = list(p[:2])
        hi, lo = oracle.split_f32c(u0)
        whi, wlo = oracle.advance_f32c(st, prm, hi, lo, nst, 1)
        seg = pool_bytes[off:off + 8 * n].view(np.float32)
        exact = exact and np.array_equal(seg[:n], whi) and np.array_equal(seg[n:], wlo)
        w64 = oracle.advance_f64(st, prm, u0, nst, 1)
        got = seg[:n].astype(np.float64) + seg[n:].astype(np.float64)
        worst = max(worst, float(np.max(np.abs(got - w64)) / np.max(np.abs(w64))))
    return {"problems": len(sub), "steps": "min(steps, 2000)", "gpu_bit_exact": bool(exact),
            "max_err_ks_f32c_vs_oracle_f64": worst}


def report_adjoint_c4(peaks, flush):
    """Gradient of J = 1/2 sum u(T)^2 for KS, N = 2^20, 20000 steps, FP64, B = 256, checkpoint
    interval at most 64 cycles; checked against finite differences along 32 seeded directions
    and against the oracle's discrete adjoint at N = 256, 500 steps.

    The finite difference is Richardson-extrapolated: with the central difference
    D(e) = (J(u0 + e v) - J(u0 - e v)) / 2e = <g, v> + c e^2 + O(e^4), the combination
    (4 D(e/2) - D(e)) / 3 cancels the e^2 term.  Over 20000 chaotic steps c is large (D(1e-6)
    is off by up to 3e-3), so the plain difference would need e near 1e-8, where rounding in
    J takes over; the extrapolation at e = 5e-7 leaves O(e^4) plus rounding."""
    import torch
    import paper_1504_01380_gb300 as sw
    n, nsteps, K, eps = 1 << 20, 20000, 64, 5e-7
    prm = [workloads.KS_DT, workloads.KS_DX]
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, prm, sw.SWEPT_F64, 256)
    u0 = torch.tensor(workloads.ks_adjoint_state(n), device="cuda")
    uT = u0.clone()
    t_fwd = cuda_time(lambda: sw.swept_advance(plan, uT, nsteps))
    g = torch.empty_like(u0)
    sw.swept_adjoint(plan, u0, uT, nsteps, K, out=g)                       # warm-up (allocates)
    torch.cuda.synchronize()
    t_grad = cuda_time(lambda: sw.swept_adjoint(plan, u0, uT, nsteps, K, out=g))
    scratch = sw.swept_adjoint_scratch(plan, nsteps, K)
    w = torch.empty_like(u0)
    jbuf = torch.empty(1, dtype=torch.float64, device="cuda")

    def J(x):
        w.copy_(x)
        sw.swept_advance(plan, w, nsteps)
        sw.swept_reduce(plan, w, sw.SWEPT_HALF_SUMSQ, out=jbuf)
        return float(jbuf.item())

    def central(v, e):
        return (J(u0 + e * v) - J(u0 - e * v)) / (2 * e)

    rich, cen, conv = [], [], []
    t0 = time.perf_counter()
    for d in range(32):
        v = torch.tensor(workloads.fd_direction(n, d), device="cuda")
        sw.swept_reduce(plan, g, sw.SWEPT_DOT, v=v, out=jbuf)
        ad = float(jbuf.item())
        d1, d2 = central(v, eps), central(v, 0.5 * eps)
        rich.append(abs((4 * d2 - d1) / 3 - ad) / abs(ad))
        cen.append(abs(d1 - ad) / abs(ad))
        conv.append(abs(d1 - ad) / max(abs(d2 - ad), 1e-300))    # the e^2 term: 4 per halving
    t_fd = time.perf_counter() - t0
    plan.destroy()
    small = cpu_leg_adjoint()
    peak, unit, source, _ = peak_block(peaks, "fp64")
    flop = 3 * ALGO_FLOP_F64["ks"] * n * nsteps
    return {"workload": "ks_adjoint_N1048576_20000steps_f64_B256_K64", "unit": "s per gradient",
            "gradient_s": t_grad, "forward_s": t_fwd, "gradient_over_forward": t_grad / t_fwd,
            "forward_equivalent_rate": n * nsteps / t_grad, "scratch_bytes": scratch,
            "fd": {"directions": 32, "eps": eps, "scheme": "Richardson (4 D(eps/2) - D(eps)) / 3 of central D",
                   "rel_err_max": max(rich), "rel_err_median": statistics.median(rich),
                   "under_1e-6": sum(r < 1e-6 for r in rich),
                   "central_rel_err_max": max(cen),
                   "central_err_ratio_eps_over_half_eps": [min(conv), max(conv)], "wall_s": t_fd},
            "roofline": roofline(flop / t_grad, peak, unit, source,
                                 kernel="gradient: forward with checkpoints + tape recompute + transposed sweep",
                                 flop_per_cell_step=3 * ALGO_FLOP_F64["ks"]),
            "oracle_check": small}


def cpu_leg_adjoint():
    """Oracle leg of the adjoint report: the oracle's discrete adjoint at N = 256, 500 steps
    against the GPU's, bit for bit and in relative max-norm (bar 1e-12)."""
    import torch
    import oracle
    import paper_1504_01380_gb300 as sw
    n, nsteps = 256, 500
    prm = [workloads.KS_DT, workloads.KS_DX]
    u0 = workloads.ks_smoothed(n, 11) * 10.0
    uT = oracle.advance_f64(oracle.KS, prm, u0, nsteps)
    t0 = time.perf_counter()
    want = oracle.adjoint_f64(oracle.KS, prm, u0, uT, nsteps)
    el = time.perf_counter() - t0
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, prm, sw.SWEPT_F64, 64)
    got = sw.swept_adjoint(plan, torch.tensor(u0, device="cuda"), torch.tensor(uT, device="cuda"),
                           nsteps, 64).cpu().numpy()
    plan.destroy()
    return {"kind": "oracle", "cores": 1, "value": n * nsteps / el, "unit": "cell-steps/s of the discrete adjoint",
            "sample": "N=256, 500 steps", "gpu_bit_exact": bool(np.array_equal(got, want)),
            "rel_max_diff": float(np.max(np.abs(got - want)) / np.max(np.abs(want)))}


# ------------------------------------------------- other workloads (lines)
def shard_problems(work, world: int):
    """Split independent problems over ranks: greedy longest-first on N*steps.

    Returns one index list per rank; every index appears exactly once.  The
    batch needs no exchange between problems, so ranks share nothing but the
    final max-time reduction.
    """
    loads = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in sorted(range(len(work)), key=lambda j: -work[j]):
        r = min(range(world), key=lambda k: (loads[k], k))
        shards[r].append(i)
        loads[r] += work[i]
    return [sorted(x) for x in shards]


def max_over_ranks(t: float, world: int, device=None) -> float:
    """Max of a per-rank time over the process group (identity for one rank)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    x = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def run_batch_workload(args):
    """4096 ragged problems (half heat, half KS), compensated FP32, one persistent launch per rank
    (the problems sharded over ranks, no exchange)."""
    import torch
    import paper_1504_01380_gb300 as sw
    from paper_1504_01380_gb300 import tune
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    kinds, lengths, steps = workloads.batch_problems()
    prm = {0: (HEAT_R, 0.0), 1: (workloads.KS_DT, workloads.KS_DX)}
    allp = [(int(k), int(n), int(s), prm[int(k)]) for k, n, s in zip(kinds, lengths, steps)]
    mine = shard_problems([n * s for _, n, s, _ in allp], world)[rank]
    problems = [allp[i] for i in mine]
    kinds, lengths, steps = kinds[mine], lengths[mine], steps[mine]
    choice = tune.tune_batch(problems, sw.SWEPT_F32C)
    batch = sw.swept_batch_plan(problems, sw.SWEPT_F32C, choice["B_heat"], choice["B_ks"])
    states = workloads.batch_initial(kinds, lengths, seed_offsets=mine)
    pool = torch.zeros(batch.pool_bytes, dtype=torch.uint8, device="cuda")
    for off, u0 in zip(batch.offsets, states):
        seg = pool[off:off + 8 * len(u0)].view(torch.float32)
        sw.swept_f32c_split(torch.tensor(u0, device="cuda"), out=seg)
    pristine = pool.clone()
    total = float(np.sum(lengths.astype(np.float64) * steps))
    for _ in range(args.warmup):
        pool.copy_(pristine)
        sw.swept_advance_batch(batch, pool)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        pool.copy_(pristine)
        ms.append(cuda_time(lambda: sw.swept_advance_batch(batch, pool)) * 1e3)
    status = sw.swept_batch_status(batch)
    t = max_over_ranks(sum(ms) / 1e3 / args.steps, world, torch.device("cuda", torch.cuda.current_device()))
    if world > 1:
        tot = torch.tensor([total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tot)
        total = float(tot.item())
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": total / t, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "dtype": "f32c", "data": "synthetic",
            "config": {"workload": "batch_4096_ragged_heat_ks_f32c", "problems": len(problems),
                       "sum_N_x_steps": total, "B_heat": choice["B_heat"], "B_ks": choice["B_ks"],
                       "tuning": choice["rates"], **batch.info()},
            "status": status}
    print(json.dumps(line), flush=True)
    return 0


def _report_line(name, fn, args):
    """Print one report as its own line (peaks measured first)."""
    import torch
    import paper_1504_01380_gb300 as sw
    sw.load()
    torch.cuda.set_device(0)
    peaks = measure_alu_peaks(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rep = fn(peaks, flush)
    print(json.dumps({"report": name, "peaks": peaks, **rep}), flush=True)
    return 0


def report_ks_rk2_f1(peaks, flush):
    """KS by the two-stage Runge-Kutta midpoint rule (two sub-timesteps with a forwarded variable,
    Section 2) from the paper's Section 6 initial condition u = 2cos(19x/128), N = 2^22, 2500
    steps (5000 sub-timesteps), FP64: swept over B in {256, 512, 1024} against the naive stepper;
    the first 100 steps against the oracle, bit for bit."""
    import torch
    import paper_1504_01380_gb300 as sw
    n, nsteps, nchk = 1 << 22, 2500, 100
    prm = [workloads.KS_DT, workloads.KS_DX]
    u0h = workloads.ks_cosine(n)
    u0 = torch.tensor(u0h, device="cuda")
    u = u0.clone()

    def run(fn):
        u.copy_(u0)
        flush.fill_(1)
        return cuda_time(fn)

    sweep = {}
    for B in (256, 512, 1024):
        plan = sw.swept_plan(n, 2, sw.SWEPT_KS_RK2, prm, sw.SWEPT_F64, B)
        run(lambda: sw.swept_advance(plan, u, nchk))
        sweep[str(B)] = n * nsteps / run(lambda: sw.swept_advance(plan, u, nsteps))
        plan.destroy()
    best = max(sweep, key=sweep.get)
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS_RK2, prm, sw.SWEPT_F64, int(best))
    naive = n * nsteps / run(lambda: sw.swept_naive_advance(plan, u, nsteps))
    run(lambda: sw.swept_advance(plan, u, nchk))
    got = u.cpu().numpy()
    plan.destroy()
    leg = cpu_leg_rk2(u0h, prm, nchk, got)
    peak, unit, source, _ = peak_block(peaks, "fp64")
    flop = 2 * ALGO_FLOP_F64["ks"]                # two KS sub-timesteps per time step
    return {"workload": f"ks_rk2_N{n}_{nsteps}steps_f64_cos19x128", "unit": UNIT + " (time steps of 2 sub-timesteps)",
            "swept": sweep[best], "best_B": int(best), "tile_sweep": sweep, "naive": naive,
            "swept_over_naive": sweep[best] / naive,
            "roofline": roofline(flop * sweep[best], peak, unit, source, kernel="swept_stream_kernel<ks_rk2,f64>",
                                 flop_per_step=flop),
            "cpu_baseline": leg}


def cpu_leg_rk2(u0, prm, nsteps, got):
    """Oracle leg of the Runge-Kutta report: the oracle's first steps on the host cores, timed,
    compared with the GPU's bit for bit."""
    import oracle
    threads = cores_used()
    t0 = time.perf_counter()
    want = oracle.advance_rk2_f64(oracle.KS_RK2, prm, u0, nsteps, threads)
    el = time.perf_counter() - t0
    return {"kind": "oracle", "cores": threads, "value": u0.size * nsteps / el, "unit": UNIT + " (time steps)",
            "sample": f"N=2^22, first {nsteps} of 2500 steps, FP64", "gpu_bit_exact": bool(np.array_equal(got, want))}


def euler_state(n: int, cfl: float = 0.2):
    """Periodic Sod state of Section 7 (rho, u, p = 0.125, 0, 0.1 | 1, 0, 1) on [0, 1), gamma 1.4,
    as planar rho/m/E; dt = cfl * dx."""
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    rho = np.where(left, 0.125, 1.0)
    E = np.where(left, 0.1, 1.0) / 0.4
    dx = 1.0 / n
    return np.concatenate([rho, np.zeros(n), E]), [cfl * dx, dx, 1.4]


def report_euler_f2(peaks, flush):
    """Euler equations (Section 7): second-order finite volumes, minmod, Roe spectral-radius
    dissipation, midpoint rule (4 sub-timesteps per step), periodic Sod state, gamma 1.4.

    For the compensated FP32 state and for FP64: throughput at N = 2^23 cells (201 MB of FP64
    state, larger than L2) over the tile widths against the naive stepper (two fused launches
    per step, one face per thread), and the latency regime at N = 4096 cells (the paper's run
    had about 50 cells on each of 64 ranks): time per sub-timestep, swept (graph-replayed
    stages) against naive (graph-replayed launches).  The 4096-cell runs are compared with the
    oracle bit for bit (both precisions), and the compensated state with the FP64 oracle."""
    import torch
    import paper_1504_01380_gb300 as sw
    out = {}
    for dtype, name, widths in ((sw.SWEPT_F32C, "f32c", (64, 128, 256)), (sw.SWEPT_F64, "f64", (32, 64, 128))):
        n, nsteps = 1 << 23, 40 if dtype == sw.SWEPT_F64 else 400
        q0, prm = euler_state(n)
        u64 = torch.tensor(q0, device="cuda")
        u0 = u64 if dtype == sw.SWEPT_F64 else sw.swept_f32c_split(u64)
        u = u0.clone()

        def mean_time(fn, reps):
            fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                u.copy_(u0)
                ts.append(cuda_time(fn))
            return sum(ts) / len(ts)

        res = {}
        for B in widths:
            plan = sw.swept_plan(n, 1, sw.SWEPT_EULER, prm, dtype, B)
            res[str(B)] = n * nsteps / mean_time(lambda: sw.swept_advance(plan, u, nsteps), 2)
            plan.destroy()
        plan = sw.swept_plan(n, 1, sw.SWEPT_EULER, prm, dtype, widths[0])
        naive = n * nsteps / mean_time(lambda: sw.swept_naive_advance(plan, u, nsteps), 2)
        plan.destroy()
        # latency regime
        nl, stl = 4096, 500
        ql, prml = euler_state(nl)
        u64 = torch.tensor(ql, device="cuda")
        u0 = u64 if dtype == sw.SWEPT_F64 else sw.swept_f32c_split(u64)
        u = u0.clone()
        lat = {}
        for B in (32, 64, 128):
            plan = sw.swept_plan(nl, 1, sw.SWEPT_EULER, prml, dtype, B)
            sw.swept_plan_set(plan, sw.SWEPT_OPT_GRAPH, 1)
            lat[str(B)] = mean_time(lambda: sw.swept_advance(plan, u, stl), 3) / (4 * stl)
            if B == 32:
                u.copy_(u0)
                sw.swept_advance(plan, u, stl)
                got = u.cpu().numpy()
            plan.destroy()
        plan = sw.swept_plan(nl, 1, sw.SWEPT_EULER, prml, dtype, 32)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sw.swept_naive_advance(plan, u, stl)
        naive_lat = mean_time(g.replay, 3) / (4 * stl)
        plan.destroy()
        best = max(res, key=res.get)
        bl = min(lat, key=lat.get)
        out[name] = {"workload": f"euler1d_sod_periodic_N{n}_{nsteps}steps_{name}_gamma1.4_cfl0.2",
                     "best_B": int(best), "swept": res[best], "tile_sweep": res, "naive": naive,
                     "swept_over_naive": res[best] / naive,
                     "latency": {"workload": f"euler1d_sod_periodic_N{nl}_{stl}steps_{name}", "best_B": int(bl),
                                 "swept_graph_ns_per_sub": {b: t * 1e9 for b, t in lat.items()},
                                 "naive_graph_ns_per_sub": naive_lat * 1e9,
                                 "speedup_vs_naive": naive_lat / lat[bl]},
                     "cpu_baseline": cpu_leg_euler(ql, prml, stl, got, dtype == sw.SWEPT_F64)}
    return {"unit": UNIT + " (time steps of 4 sub-timesteps)", **out}


def cpu_leg_euler(q_planar, prm, nsteps, got, fp64: bool):
    """Oracle leg of the Euler report: the oracle (FP64 or compensated FP32) on the 4096-cell
    latency workload, timed on one core, compared with the GPU's bit for bit; the compensated
    result's error against the FP64 oracle."""
    import oracle
    n = q_planar.size // 3
    q = q_planar.reshape(3, n).T.copy()                      # (N, 3) rows of (rho, m, E)
    t0 = time.perf_counter()
    if fp64:
        want = oracle.euler_advance(prm, q, nsteps)
        el = time.perf_counter() - t0
        exact = bool(np.array_equal(got.reshape(3, n).T, want))
        err = None
    else:
        hi, lo = oracle.split_f32c(q.reshape(-1))
        whi, wlo = oracle.euler_advance_f32c(prm, hi.reshape(-1, 3), lo.reshape(-1, 3), nsteps)
        el = time.perf_counter() - t0
        ghi = got[:3 * n].reshape(3, n).T
        glo = got[3 * n:].reshape(3, n).T
        exact = bool(np.array_equal(ghi, whi) and np.array_equal(glo, wlo))
        w64 = oracle.euler_advance(prm, q, nsteps)
        val = ghi.astype(np.float64) + glo.astype(np.float64)
        err = float(np.max(np.abs(val - w64)) / np.max(np.abs(w64)))
    return {"kind": "oracle", "cores": 1, "value": n * nsteps / el, "unit": "cell-steps/s",
            "sample": f"the {n}-cell latency workload, {nsteps} steps", "gpu_bit_exact": exact,
            "max_err_f32c_vs_oracle_f64": err}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--reports", default="all", choices=["all", "none"],
                    help="one GPU: the other workloads' reports after the headline (all), or the "
                         "headline line alone (none; e.g. for a launch list of the headline steps)")
    ap.add_argument("--workload", default="heat",
                    choices=["heat", "ks", "batch", "adjoint", "latency", "heat_f64", "ks_rk2", "euler", "uneven"],
                    help="heat: the headline line (with every report on one GPU); the others print one "
                         "line for that workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch_workload(args)
    reports = {"ks": ("ks_c2", report_ks_c2), "adjoint": ("adjoint_c4", report_adjoint_c4),
               "latency": ("latency_c0", report_latency_c0), "heat_f64": ("heat_c1_f64", report_heat_f64),
               "ks_rk2": ("ks_rk2_f1", report_ks_rk2_f1), "euler": ("euler_f2", report_euler_f2),
               "uneven": ("uneven_f4", report_uneven_f4)}
    if args.workload in reports:
        return _report_line(*reports[args.workload], args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
