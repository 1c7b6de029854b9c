"""Autotuner: picks a built tile width, caches it, and its choice runs bit-exact."""
from __future__ import annotations

import json

import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_tune_single_and_cache(cuda_lib, tmp_path, monkeypatch):
    sw = cuda_lib
    from paper_1504_01380_gb300 import tune
    monkeypatch.setenv("SWEPT_TUNE_CACHE", str(tmp_path / "tune.json"))
    res = tune.tune_single(1 << 18, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F32C, stages=3, reps=1)
    assert res["B"] in tune.CANDIDATE_B
    assert len(res["rates"]) == len(tune.CANDIDATE_B)
    cached = json.load(open(tmp_path / "tune.json"))
    assert len(cached) == 1 and list(cached.values())[0]["B"] == res["B"]
    assert tune.best_B(1 << 18, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F32C) == res["B"]   # from the cache


def test_tune_batch(cuda_lib):
    sw = cuda_lib
    from paper_1504_01380_gb300 import tune
    kinds, lengths, steps = workloads.batch_problems(64, 512, 16384, 100, 600)
    prm = {0: (0.25, 0.0), 1: (workloads.KS_DT, workloads.KS_DX)}
    problems = [(int(k), int(n), int(s), prm[int(k)]) for k, n, s in zip(kinds, lengths, steps)]
    res = tune.tune_batch(problems, sw.SWEPT_F32C)
    assert (res["B_heat"], res["B_ks"]) in [(256, 256), (256, 512), (512, 256), (512, 512)]
