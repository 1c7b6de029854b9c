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
