"""Host logic of bench.py (no GPU): the nvidia-smi clock sampler against a
fake nvidia-smi on PATH (median and maximum SM clock of the sampled GPU only,
throttle reasons seen while it ran, the unavailable case), the roofline peaks
(measured file, else the stated fallback), and the DRAM-traffic figure that
is given only while the product's sources match the profiled ones."""
import json
import os
import stat
import time

import bench

FAKE = """#!/bin/sh
printf '%s\\n' \\
 '0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active' \\
 '1, 900, 2070, 400.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active' \\
 '0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active' \\
 '0, 2070, 2070, 1101.7, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active' \\
 'garbage line'
exec sleep 30
"""


def _fake_smi(tmp_path):
    path = tmp_path / "nvidia-smi"
    path.write_text(FAKE)
    path.chmod(path.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def _sample(gpu):
    s = bench.ClockSampler(gpu)
    s.start()
    deadline = time.time() + 10
    while len(s.rows) < 4 and time.time() < deadline:
        time.sleep(0.05)
    return s.stop()


def test_clock_sampler_reads_its_own_gpu(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path) + os.pathsep + os.environ["PATH"])
    c = _sample(0)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    c = _sample(1)
    assert c["samples"] == 1 and c["sm_mhz"] == 900.0
    assert c["reasons"] == ["hw_slowdown"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_measured_peaks_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, how = bench.measured_peaks()
    assert how == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6794.1, "bf16_tflops": 1884.0}))
    peaks, how = bench.measured_peaks()
    assert how == "measured" and peaks["hbm_gbs"] == 6794.1


def test_traffic_only_for_the_profiled_sources(tmp_path, monkeypatch):
    t = bench.apply_traffic()
    assert isinstance(t, int) and t > 303038464      # DRAM bytes exceed the algorithmic ones
    assert bench.apply_traffic(bench.synth.W3D_N128) is None
    changed = tmp_path / "apply_impl.cuh"
    changed.write_text("// a changed kernel source\n")
    monkeypatch.setattr(bench, "APPLY_SOURCES", [str(changed)])
    assert bench.apply_traffic() is None
