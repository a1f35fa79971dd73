"""bench.py's host-side bookkeeping (no GPU): the clock record that decides whether
a timed run is kept, and the HBM peak the roofline divides by."""
import json
import os

import pytest

import bench


def _summary_of(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(l + "\n" for l in lines))
    s = bench.ClockSampler(0)
    s.proc, s.path = object(), str(path)
    return s.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    ok = "0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"
    lines = [ok.format(mhz=m, cap="Not Active") for m in (2070, 2055, 2070, 1980)]
    lines.append(ok.format(mhz=1900, cap="Active"))
    lines.append("garbage line")
    s = _summary_of(tmp_path, lines)
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 5
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_and_hw_slowdown(tmp_path):
    line = "0, 1500, 2070, 1300.0, 0x48, Active, Not Active, Active, Not Active"
    s = _summary_of(tmp_path, [line])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_reads_the_hbm_clock_and_temperature(tmp_path):
    ok = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    mem = tmp_path / "mem.csv"
    mem.write_text("3996, 3996, 51\n3200, 3996, 58\n3996, 3996, N/A\nbad line\n")
    path = tmp_path / "clocks.csv"
    path.write_text(ok + "\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = object(), str(path)
    s.mem_proc, s.mem_path = object(), str(mem)
    r = s.summary()
    assert r["sm_mhz"] == 2070 and r["mem_mhz"] == 3996 and r["mem_max_mhz"] == 3996
    assert r["mem_temp_c_max"] == 58
    # no memory record: the SM record stands alone
    assert _summary_of(tmp_path, [ok])["mem_mhz"] is None


def test_clock_summary_without_nvidia_smi(monkeypatch, tmp_path):
    s = bench.ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]
    # a sampler whose nvidia-smi cannot start leaves no record file behind
    import subprocess
    import tempfile

    def no_smi(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(subprocess, "Popen", no_smi)
    monkeypatch.setattr(tempfile, "tempdir", str(tmp_path))
    with bench.ClockSampler(0) as cs:
        pass
    assert cs.summary()["reasons"] == ["nvidia-smi unavailable"]
    assert list(tmp_path.iterdir()) == []


def test_peak_is_the_measured_copy_bandwidth_else_the_fallback(monkeypatch, tmp_path):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6753.8}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6753.8, "measured")
    os.unlink(tmp_path / "MEASURED_PEAKS.json")
    assert bench.peaks() == (pytest.approx(6800.0), "fallback")


def test_traffic_key_ignores_comments_but_not_code():
    src = {rel: open(os.path.join(bench.ROOT, rel)).read() for rel in bench.FUSED_SOURCES}
    base = bench.fused_source_hash(src.__getitem__)
    assert base == bench.fused_source_hash()
    first = bench.FUSED_SOURCES[0]
    commented = dict(src)
    commented[first] = "// a note\n/* a block\n   comment */\n" + src[first].replace("\n", "  // tail\n", 3)
    assert bench.fused_source_hash(commented.__getitem__) == base
    edited = dict(src)
    edited[first] = src[first] + "\nstatic const int k_extra = 1;\n"
    assert bench.fused_source_hash(edited.__getitem__) != base
