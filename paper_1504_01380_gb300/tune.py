"""Autotuner for the swept launch: tile width B and ring warp count, timed on the GPU.

Section 4 models the time per sub-timestep of a node owning n points as
n*s + 2*tau/n (s: time of one point-update, tau: latency of one exchange),
minimised at n* = sqrt(2 tau / s).  On the GPU the "node" is a warp, tau is
the per-stage cost that does not scale with the tile (edge load/store, the
first and last half-slot of a run, the launch) and s the cost of a point
update; both are measured here by timing swept_advance over a few stages for
each candidate B, and the fit of the model to the measurements is returned
with the choice.  Results are cached per (GPU, stencil, dtype, log2 N) in a
JSON file ($SWEPT_TUNE_CACHE, default ~/.cache/swept/tune.json).
"""
from __future__ import annotations

import json
import math
import os

from . import (SWEPT_DIAMOND_RING, SWEPT_F32C, SWEPT_HEAT, SWEPT_OPT_DIAMOND, SWEPT_OPT_RING_WARPS,
               RADIUS, swept_advance, swept_plan, swept_plan_set)

CANDIDATE_B = (64, 128, 256, 512, 1024)


def cache_path() -> str:
    return os.environ.get("SWEPT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "swept", "tune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(c: dict):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _key(stencil: int, dtype: int, N: int) -> str:
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|st{stencil}|dt{dtype}|log2N{int(round(math.log2(N)))}"


def fit_eq1(points):
    """Least-squares fit of t = n*s + c/n (c = 2 tau) to [(n, t)]; returns s, tau, n*."""
    # normal equations for t = s*n + c*(1/n)
    a11 = sum(n * n for n, _ in points)
    a12 = sum(1.0 for _ in points)
    a22 = sum(1.0 / (n * n) for n, _ in points)
    b1 = sum(n * t for n, t in points)
    b2 = sum(t / n for n, t in points)
    det = a11 * a22 - a12 * a12
    if det == 0:
        return None
    s = (b1 * a22 - b2 * a12) / det
    c = (a11 * b2 - a12 * b1) / det
    nstar = math.sqrt(c / s) if s > 0 and c > 0 else None
    return {"s": s, "tau": c / 2.0, "n_star": nstar}


def tune_single(N: int, stencil: int, params, dtype: int = SWEPT_F32C, stages: int = 6, reps: int = 2,
                candidates=CANDIDATE_B, ring_warps=(0,), use_cache: bool = True) -> dict:
    """Time swept_advance for every candidate (B, ring warps) and pick the fastest.

    Returns {"B", "ring_warps", "rates": {B: cell-updates/s}, "model": fit}.
    """
    import torch
    key = _key(stencil, dtype, N)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    r = RADIUS[stencil]
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    if dtype == SWEPT_F32C:
        u = torch.zeros(2 * N, dtype=torch.float32, device="cuda")
    u.normal_()
    rates, times, best = {}, [], None
    for B in candidates:
        K = B // 32
        if K % r or N % B or B > N:
            continue
        plan = swept_plan(N, r, stencil, params, dtype, B)
        nsteps = stages * plan.h
        for w in ring_warps:
            swept_plan_set(plan, SWEPT_OPT_DIAMOND, SWEPT_DIAMOND_RING)
            swept_plan_set(plan, SWEPT_OPT_RING_WARPS, w)
            swept_advance(plan, u, nsteps)          # warm-up
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(reps):
                swept_advance(plan, u, nsteps)
            ev[1].record()
            torch.cuda.synchronize()
            sec = ev[0].elapsed_time(ev[1]) / 1e3 / reps
            rate = N * nsteps / sec
            rates[f"{B}/{w}"] = rate
            if best is None or rate > best[0]:
                best = (rate, B, w)
        # time of one level of one window (n = B points), up to the constant
        # number of windows in flight: B / (cell-updates per second)
        times.append((B, B / max(rates[f"{B}/{w}"] for w in ring_warps)))
        plan.destroy()
    out = {"B": best[1], "ring_warps": best[2], "rates": rates, "model": fit_eq1(times)}
    if use_cache:
        cache[key] = out
        _store_cache(cache)
    return out


def best_B(N: int, stencil: int, params, dtype: int = SWEPT_F32C) -> int:
    """Tuned tile width for this size class (tunes and caches on first use)."""
    return int(tune_single(N, stencil, params, dtype)["B"])


def tune_batch(problems, dtype: int = SWEPT_F32C, sample: int = 256, seed: int = 0,
               candidates=((256, 256), (256, 512), (512, 256), (512, 512))) -> dict:
    """Pick (B_heat, B_ks) for a batch by timing swept_advance_batch on a sample of it."""
    import random

    import torch

    from . import swept_advance_batch, swept_batch_plan
    rnd = random.Random(seed)
    sub = problems if len(problems) <= sample else rnd.sample(list(problems), sample)
    rates = {}
    for bh, bk in candidates:
        ok = [p for p in sub if p[1] % (bh if p[0] == SWEPT_HEAT else bk) == 0]
        if len(ok) < len(sub):
            continue
        batch = swept_batch_plan(sub, dtype, bh, bk)
        pool = torch.zeros(batch.pool_bytes, dtype=torch.uint8, device="cuda")
        swept_advance_batch(batch, pool)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        swept_advance_batch(batch, pool)
        ev[1].record()
        torch.cuda.synchronize()
        sec = ev[0].elapsed_time(ev[1]) / 1e3
        rates[f"{bh}/{bk}"] = sum(n * s for _, n, s, _ in sub) / sec
        batch.destroy()
    best = max(rates, key=rates.get)
    bh, bk = (int(x) for x in best.split("/"))
    return {"B_heat": bh, "B_ks": bk, "rates": rates}
