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


def test_serving_result_ring_keeps_every_array_aligned():
    """The serving client's ring of page-locked result buffers: every array of
    every slot at a multiple of its element size and inside its slot, for the
    largest event and smaller ones (an odd largest track count once gave slots
    4 bytes off an 8-byte boundary; the server now stages such arrays, and the
    ring no longer produces them)."""
    import numpy as np
    for max_n, L in ((47015, 17), (50000, 17), (1, 4), (12345, 9)):
        per = bench.result_slot_bytes(max_n, L)
        assert per % 64 == 0
        ring = 5
        raw = np.zeros(per * ring + 64, np.uint8)
        base = (-raw.ctypes.data) % 64
        buf = raw[base:base + per * ring]
        for slot in range(ring):
            for n in (max_n, max(1, max_n // 3), 1):
                views = bench.result_views(buf, per, slot, n, L)
                assert [k for k, _, _ in bench.result_arrays_layout(n, L)] == list(views)
                ends = []
                for k, a in views.items():
                    assert a.flags.aligned and a.ctypes.data % a.dtype.itemsize == 0, (max_n, L, slot, n, k)
                    off = a.ctypes.data - buf.ctypes.data
                    assert slot * per <= off and off + a.nbytes <= (slot + 1) * per
                    ends.append((off, off + a.nbytes))
                ends.sort()
                assert all(e0[1] <= e1[0] for e0, e1 in zip(ends, ends[1:]))  # no overlap
