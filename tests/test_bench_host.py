"""Host logic of bench.py that needs no GPU: the clock record taken during the timed region
(median SM clock under load, throttle reasons) and the roofline denominators."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _record(tmp_path, lines):
    c = bench.Clocks(0)
    p = tmp_path / "clocks.csv"
    p.write_text("".join(line + "\n" for line in lines))
    c.proc, c.path = _DoneProc(), str(p)
    return c.stop()


def test_clock_record_median_and_reasons(tmp_path):
    rows = ["0, 2070, 2070, 901.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1200.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1390.9, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "garbage line",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    r = _record(tmp_path, rows)
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]  # kept and noted; a slowdown reason rejects a run
    r = _record(tmp_path, ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active"])
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_sampler():
    assert bench.Clocks(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_are_the_measured_ones_when_present():
    p, note = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert note == "of measured" and p["hbm_gbs"] > 1000
    else:
        assert note == "of fallback" and p["hbm_gbs"] == 6800.0
