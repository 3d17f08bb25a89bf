"""Host logic of bench.py that needs no GPU: algorithmic bytes, the peak it
reports against, and the clock sampler's reading of nvidia-smi output (fed by
a stand-in nvidia-smi on PATH)."""
import importlib.util
import json
import os
import stat
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_of_the_live_view_stack(bench):
    cfg = bench.opm_synth.CONFIGS["liveview_200x512x2048"]
    live, vol = bench.algorithmic_bytes(cfg, 1021)
    raw = 200 * 512 * 2048 * 2
    assert live == raw + 1021 * 2048 * 4 + 512 * 2048 * 4 == 431_988_736
    assert vol == raw + 512 * 1021 * 2048 * 4 == 4_701_814_784


def test_peak_is_the_measured_copy_bandwidth(bench):
    peak, src = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert (peak, src) == (float(json.load(f)["hbm_gbs"]), "measured")
    else:
        assert (peak, src) == (6800.0, "fallback")


def _fake_smi(tmp_path, lines):
    exe = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{ln}'" for ln in lines)
    exe.write_text(f"#!/bin/sh\n{body}\nsleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


@pytest.mark.parametrize("rows,want_reasons,want_sm", [
    (["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"] * 3, [], 2070.0),
    (["0, 1500, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
      "0, 1700, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
      "0, 1900, 2070, 1390.0, 0x0, Not Active, Not Active, Not Active, Not Active"], ["sw_power_cap"], 1700.0),
    (["0, 900, 2070, 500.0, 0x8, Active, Not Active, Not Active, Not Active"], ["hw_slowdown"], 900.0),
])
def test_clock_sampler_reads_clocks_and_reasons(bench, tmp_path, monkeypatch, rows, want_reasons, want_sm):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert out["sm_mhz"] == want_sm and out["sm_max_mhz"] == 2070.0
    assert out["samples"] == len(rows) and out["reasons"] == want_reasons


def test_clock_sampler_without_nvidia_smi(bench, tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
