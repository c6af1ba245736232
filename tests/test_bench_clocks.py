"""The bench's clock record: parsing of the nvidia-smi samples taken during
the timed region (median SM clock, maximum, throttle reasons seen), and the
record of a run where no sample could be taken."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.5", "0x0000000000000000", hw, hwt, swt, cap]


def test_summary_median_max_and_reasons():
    import bench
    c = bench.ClockSampler()
    c.samples = [_line(2070, 2070), _line(1995, 2070, cap="Active"), _line(2070, 2070),
                 _line(1800, 2070, hwt="Active"), ["garbled"]]
    s = c.summary()
    assert s["sm_mhz"] == 2032.5 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["samples"] == 5


def test_unsampled_run_is_marked():
    import bench
    c = bench.ClockSampler()
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_sampler_without_nvidia_smi_is_harmless(monkeypatch):
    import bench
    monkeypatch.setenv("PATH", "/nonexistent")
    with bench.ClockSampler() as c:
        pass
    assert c.proc is None and c.summary()["reasons"] == ["unsampled"]
