"""Host-side logic of bench.py that needs no GPU: the clock sampler that runs
nvidia-smi beside the timed region, driven here by a stand-in script."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


ROWS = ("0, 1965, 2070, 812.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 905.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1120.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n")


def test_parse_median_max_and_reasons():
    d = bench.ClockSampler.parse(ROWS + "0, 2010, 20")  # last row cut short
    assert d["samples"] == 3
    assert d["sm_mhz"] == 1980.0 and d["sm_max_mhz"] == 2070.0
    assert d["reasons"] == ["sw_power_cap"]


def test_parse_unavailable_fields_and_empty_output():
    d = bench.ClockSampler.parse("0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n")
    assert d == dict(sm_mhz=None, sm_max_mhz=None, samples=1, reasons=[])
    assert bench.ClockSampler.parse("") is None
    assert bench.ClockSampler.parse("garbage\n") is None


def test_sampler_runs_a_stand_in_nvidia_smi(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\ncat <<'X'\n" + ROWS + "X\nexec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    d = s.stop()
    assert d["samples"] == 3 and d["reasons"] == ["sw_power_cap"] and d["sm_mhz"] == 1980.0


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() is None
