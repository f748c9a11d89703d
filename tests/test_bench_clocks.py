"""The benchmark's clock record: nvidia-smi samples taken during the timed
region are summarised as the median SM clock, the maximum clock and every
throttle reason seen active (a run with hw_slowdown, hw_thermal_slowdown or
sw_thermal_slowdown is rejected; sw_power_cap is kept and noted). CPU only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

NA = "Not Active"


def line(sm, mx, pw, hw=NA, hwt=NA, swt=NA, cap=NA):
    return f"{sm}, {mx}, {pw}, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_clean_run():
    out = bench.ClockSampler.summarise([line(2070, 2070, 600.5), line(2070, 2070, 655.2), line(1995, 2070, 640.0)])
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 3 and out["power_w_max"] == 655.2


def test_reasons_seen_in_any_sample():
    out = bench.ClockSampler.summarise([line(2070, 2070, 900.0), line(1800, 2070, 1400.0, cap="Active"),
                                        line(1500, 2070, 1390.0, hwt="Active")])
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1800.0


def test_malformed_and_missing_samples():
    out = bench.ClockSampler.summarise(["garbage\n", line("[N/A]", 2070, "[N/A]"), line(2070, 2070, 700.0)])
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0 and out["power_w_max"] == 700.0
    assert bench.ClockSampler.summarise([])["reasons"] == ["no samples"]


def test_stop_reads_the_samples_and_removes_the_file():
    """stop() ends the sampling process, reads its file and deletes it (a
    sleeping Python process stands in for nvidia-smi)."""
    import subprocess
    s = bench.ClockSampler(None)
    s.f = open(s.path, "w")
    s.f.write(line(2070, 2070, 610.0) + line(2070, 2070, 620.0))
    s.f.flush()
    s.proc = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(60)"])
    out = s.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    assert not os.path.exists(s.path)
    assert s.proc.poll() is not None


def test_unavailable_sampler_leaves_no_file():
    s = bench.ClockSampler(None)
    s.proc = None
    out = s.stop()
    assert out["reasons"] == ["nvidia-smi unavailable"] and not os.path.exists(s.path)
