"""Host logic of bench.py, without a GPU: the clock sampler keeps only the
samples taken inside the timed region (a fake nvidia-smi on PATH prints one
throttled line before the region, unthrottled ones after), and the DRAM
traffic figure of the committed ncu summary is used only while the kernel
sources it was captured from are unchanged."""
import importlib.util
import json
import os
import stat
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


FAKE_SMI = """#!/bin/bash
echo "0, 1000, 2070, 100.0, 0x08, Active, Not Active, Not Active, Not Active"
while true; do
  sleep 0.05
  echo "0, 2070, 2070, 900.0, 0x04, Not Active, Not Active, Not Active, Active"
done
"""


def test_clock_sampler_keeps_the_timed_region_only(monkeypatch):
    b = _bench()
    d = tempfile.mkdtemp(prefix="fake_smi_")
    path = os.path.join(d, "nvidia-smi")
    with open(path, "w") as f:
        f.write(FAKE_SMI)
    os.chmod(path, os.stat(path).st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    s = b.ClockSampler(0)
    s.start()
    time.sleep(0.4)
    clk = s.stop()
    assert clk is not None and clk["samples"] >= 2
    assert clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]  # the throttled line came before the region
    assert "sampled_just_before_region" not in clk


def test_clock_sampler_without_nvidia_smi_reports_nothing(monkeypatch):
    b = _bench()
    monkeypatch.setenv("PATH", tempfile.mkdtemp(prefix="empty_path_"))
    s = b.ClockSampler(0)
    s.start()
    assert s.stop() is None


def test_traffic_figure_follows_the_kernel_sources(monkeypatch):
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "k_image_sched_180_traffic.json")) as f:
        d = json.load(f)
    if d["csrc_sha"] == b.kernel_source_hash():
        assert b.ncu_traffic() == float(d["dram_bytes_per_layer"])
    else:  # sources changed since the capture: the bench reports no traffic
        assert b.ncu_traffic() is None
    monkeypatch.setattr(b, "kernel_source_hash", lambda: d["csrc_sha"])
    assert b.ncu_traffic() == float(d["dram_bytes_per_layer"])
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "0" * 16)
    assert b.ncu_traffic() is None
