"""Host logic of bench.py that needs no GPU: the parsing of the nvidia-smi
clock samples (median SM clock, throttle reasons) and the error figures
reported beside the throughput."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class FakeSmi:
    """Stands in for the nvidia-smi process: returns canned CSV lines."""

    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def sampled(lines):
    s = bench.ClockSampler(0)
    s.proc = FakeSmi("\n".join(lines) + "\n")
    return s.stop()


NA = "Not Active"


def test_clock_samples_median_max_and_power_cap():
    r = sampled([
        "0, 2070, 2070, 900.5, 0x0, %s, %s, %s, %s" % (NA, NA, NA, NA),
        "0, 2055, 2070, 1300.0, 0x4, %s, %s, %s, Active" % (NA, NA, NA),
        "0, 1980, 2070, 1390.0, 0x4, %s, %s, %s, Active" % (NA, NA, NA),
    ])
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_samples_report_thermal_and_hw_slowdown():
    r = sampled([
        "0, 1500, 2070, 1000.0, 0x48, Active, %s, %s, %s" % (NA, NA, NA),
        "0, 1400, 2070, 1000.0, 0x48, %s, Active, Active, %s" % (NA, NA),
    ])
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1450.0


def test_clock_samples_skip_malformed_lines():
    r = sampled(["[N/A], [N/A]", "garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d"])
    assert r["sm_mhz"] is None and r["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_error_figures():
    rng = np.random.default_rng(4)
    u_ref = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    g_ref = rng.standard_normal((64, 2)) + 1j * rng.standard_normal((64, 2))
    du = np.zeros(64, complex)
    du[5] = 1e-3
    dg = np.zeros((64, 2), complex)
    dg[7] = (3e-4, 4e-4j)
    e = bench.errors(u_ref + du, g_ref + dg, u_ref, g_ref)
    assert np.isclose(e["pot"], 1e-3 / np.linalg.norm(u_ref))
    assert np.isclose(e["grad"], 5e-4 / np.linalg.norm(g_ref))
    rms_u = np.sqrt(np.mean(np.abs(u_ref) ** 2))
    rms_g = np.sqrt(np.mean(np.sum(np.abs(g_ref) ** 2, axis=1)))
    assert np.isclose(e["pot_max_over_rms"], 1e-3 / rms_u)
    assert np.isclose(e["grad_max_over_rms"], 5e-4 / rms_g)
