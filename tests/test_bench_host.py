"""Host logic of bench.py that decides what a result line may claim: the
clock record (median SM clock and the throttle reasons that reject a run)
parsed from the nvidia-smi samples, and the DRAM traffic taken from a
committed ncu summary only while the kernel source it was measured on is
unchanged."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(tmp_path, lines):
    """An nvidia-smi stand-in on PATH that prints the given CSV samples."""
    d = tmp_path / "bin"
    d.mkdir()
    script = d / "nvidia-smi"
    body = "\n".join(f"echo '{ln}'" for ln in lines)
    script.write_text("#!/bin/sh\n" + body + "\nexec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(d)


def test_clock_record_median_and_reasons(tmp_path, monkeypatch):
    lines = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2055, 2070, 1201.0, 0x4, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 1250.5, 0x4, Not Active, Not Active, Not Active, Active",
             "garbage line",
             "1980, 2070, 1300.0, 0x20, Not Active, Not Active, Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0)
    time.sleep(1.0)
    rec = cs.stop()
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == pytest.approx(2062.5)
    assert rec["sm_max_mhz"] == 2070.0
    # sw_power_cap is kept and noted; a thermal slowdown rejects the run
    assert rec["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    assert not os.path.exists(cs.path)


def test_clock_record_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    rec = cs.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(cs.path)


def test_profiled_traffic_only_for_the_current_kernel_source(tmp_path):
    good = tmp_path / "good.md"
    good.write_text(f"kernel_source_sha: `{bench.kernel_source_hash()}`\n"
                    "dram_bytes_per_launch: 612458496\ndram_bytes_per_lu: 155.62\n")
    assert bench.profiled_traffic(str(good)) == 612458496.0
    assert bench.profiled_traffic(str(good), key="dram_bytes_per_lu") == 155.62
    stale = tmp_path / "stale.md"
    stale.write_text("kernel_source_sha: `0123456789abcdef`\ndram_bytes_per_launch: 612458496\n")
    assert bench.profiled_traffic(str(stale)) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md")) is None
    # the committed summaries carry the key the bench reads
    for name, key in (("step_d3q19_f32_128cube.md", "dram_bytes_per_launch"),
                      ("batch_step_d2q9_f32_64grids.md", "dram_bytes_per_lu")):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "kernel_source_sha:" in text and key + ":" in text


def test_whole_job_throughput_counts_every_rank():
    assert bench.whole_job_glups(2_097_152, 100, 4, 0.5) == pytest.approx(2_097_152 * 100 * 4 / 0.5 / 1e9)
