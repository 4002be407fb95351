"""Host-side measurement logic of bench.py (CPU): the clock sampler that
records SM clocks and throttle reasons during the timed region."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.rows = [["2070", "2070", "900.5", "Not Active", "Not Active", "Not Active", "Active"],
              ["1980", "2070", "1390.1", "Not Active", "Not Active", "Not Active", "Active"],
              ["2040", "2070", "1100.0", "Not Active", "Active", "Not Active", "Not Active"],
              ["[N/A]", "2070", "[N/A]", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0            # median of the three readable samples
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["samples"] == 4


def test_clock_summary_without_samples_is_none():
    assert bench.Clocks(0).summary() is None


def test_clock_sampler_reads_nvidia_smi_output(tmp_path, monkeypatch):
    """A stand-in nvidia-smi on PATH prints CSV rows; the sampler started
    around a region collects them and ends the process on exit."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "while true; do\n"
                    "  echo '2070, 2070, 1000.00, Not Active, Not Active, Not Active, Not Active'\n"
                    "  sleep 0.05\n"
                    "done\n")
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    with bench.Clocks(0) as clk:
        deadline = time.time() + 10
        while not clk.rows and time.time() < deadline:
            time.sleep(0.05)
    assert clk.proc.poll() is not None      # the sampler process has ended
    s = clk.summary()
    assert s["sm_mhz"] == 2070.0 and s["reasons"] == [] and s["samples"] >= 1


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))   # no nvidia-smi anywhere on PATH
    with bench.Clocks(0) as clk:
        pass
    assert clk.proc is None and clk.summary() is None
