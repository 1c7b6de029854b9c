"""Host-side logic of bench.py that decides whether a timing is valid: the clock record
taken during the timed region (throttle reasons, median SM clock) and the peak fallback."""
from __future__ import annotations

import bench


class _Running:
    """Stands in for the nvidia-smi process once it has been stopped."""


def _summary(lines, tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(line + "\n" for line in lines))
    cs = bench.ClockSampler(0)
    cs.proc = _Running()
    cs.path = str(p)
    return cs.summary()


ROW = "0, {sm}, 2070, 900.5 W, {act}, {hw}, {hwt}, {swt}, {cap}"


def row(sm=2070, act="0x0", hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ROW.format(sm=sm, act=act, hw=hw, hwt=hwt, swt=swt, cap=cap)


def test_clean_run(tmp_path):
    s = _summary([row(), row(sm=2055), row()], tmp_path)
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == []


def test_throttle_reasons_are_reported(tmp_path):
    s = _summary([row(), row(sm=1800, hwt="Active"), row(cap="Active")], tmp_path)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_unparsable_and_short_lines_are_skipped(tmp_path):
    s = _summary(["garbage", "0, [N/A], 2070, 1 W, 0x0, Not Active, Not Active, Not Active, Not Active",
                  row(sm=1990)], tmp_path)
    assert s["samples"] == 1 and s["sm_mhz"] == 1990


def test_no_samples_and_no_tool(tmp_path):
    assert _summary([], tmp_path)["reasons"] == ["no samples"]
    cs = bench.ClockSampler(0)                       # never started: nvidia-smi missing
    assert cs.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_peak_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))          # no MEASURED_PEAKS.json there
    assert bench.measured_hbm_gbs() == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6793.2}')
    assert bench.measured_hbm_gbs() == 6793.2


def test_traffic_only_from_a_capture_of_the_current_sources(monkeypatch, tmp_path):
    """The roofline's DRAM traffic comes from a committed ncu summary only while the kernel
    sources it was captured from are unchanged (their digest is written in the summary)."""
    csrc = tmp_path / "paper_1504_01380_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "p.md"
    assert bench.profile_traffic(str(prof), ("a.cuh",))[0] is None            # no file
    digest = bench.source_digest(("a.cuh",))
    body = ("- dram__bytes_read.sum = 10.5 Gbyte\n- dram__bytes_write.sum = 2.25 Gbyte\n")
    prof.write_text(body)
    assert bench.profile_traffic(str(prof), ("a.cuh",))[0] is None            # no digest recorded
    prof.write_text(f"source digest: `{digest}`\n" + body)
    t, note = bench.profile_traffic(str(prof), ("a.cuh",))
    assert t == 12.75e9 and "current" in note
    (csrc / "a.cuh").write_text("kernel  v1 // a note\n/* and\n another */")  # comments only
    assert bench.profile_traffic(str(prof), ("a.cuh",))[0] == 12.75e9
    (csrc / "a.cuh").write_text("kernel v2")                                  # the kernel changed
    t, note = bench.profile_traffic(str(prof), ("a.cuh",))
    assert t is None and "changed" in note


def test_code_tokens_strips_comments_not_strings():
    src = 'int a = 1; // one\n/* two\n lines */ const char* s = "// kept /* too */";\n  int  b;'
    assert bench.code_tokens(src) == 'int a = 1; const char* s = "// kept /* too */"; int b;'


def test_alu_peak_fallback_is_the_nominal_rate(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, unit, source, nominal = bench.peak_block(None, "fp32")
    assert peak == nominal == 152 * 128 * 2070e6 and source.startswith("nominal")
    measured = {"fp32_ops_per_s": 38e12, "f32_fma": {"sm_mhz": 2070},
                "fp64_flop_per_s": 1.2e12, "f64_fma": {"sm_mhz": 2070}}
    assert bench.peak_block(measured, "fp32")[0] == 38e12
    assert bench.peak_block(measured, "fp64")[0] == 1.2e12
    assert bench.peak_block(None, "fp64")[0] is None
    r = bench.roofline(19e12, 38e12, "FP32 ops/s", "measured")
    assert r["frac"] == 0.5 and r["achieved"] == 19.0 and r["peak"] == 38.0


def test_exact_heat_closed_form():
    """The bench's error reference: a single Fourier mode is scaled by g_k^n, and the mean is kept."""
    import numpy as np
    n, k, r, steps = 64, 3, 0.25, 37
    x = np.arange(n)
    u0 = 2.0 + np.sin(2 * np.pi * k * x / n)
    g = 1 - 4 * r * np.sin(np.pi * k / n) ** 2
    want = 2.0 + g ** steps * np.sin(2 * np.pi * k * x / n)
    assert np.max(np.abs(bench.exact_heat(u0, r, steps) - want)) < 1e-13
