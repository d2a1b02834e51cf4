"""Host logic of bench.py that needs no GPU: the clock, power and throttle record of the timed region."""
import bench


class _FakeSmi:
    """Stands in for the nvidia-smi sampling process: the lines it would have printed."""

    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.proc = _FakeSmi("\n".join(lines) + "\n")
    return c


def test_clock_record_medians_power_and_reasons():
    lines = [
        # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
        "0, 1650, 2070, 1360.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1640, 2070, 1370.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1700, 2070, 1340.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 1650.0
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["power_w"] == 1360.5
    assert rec["power_w_max"] == 1370.0


def test_clock_record_flags_thermal_slowdown_and_tolerates_missing_power():
    lines = ["0, 1200, 2070, [N/A], 0x20, Not Active, Active, Not Active, Not Active",
             "0, 1210, 2070, [N/A], 0x20, Not Active, Active, Not Active, Not Active"]
    rec = _sampler(lines).stop()
    assert rec["reasons"] == ["hw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1205.0
    assert "power_w" not in rec


def test_clock_record_without_samples_is_none():
    assert _sampler([]).stop() is None
    assert bench.ClockSampler(0).stop() is None
