"""Host logic of the benchmark that needs no GPU: the clock sampler keeps only
the nvidia-smi lines that arrive inside the timed region, and reads the
throttle reasons from them."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _line(mhz, hw="Not Active", power_cap="Not Active"):
    return f"0, {mhz}, 2070, 950.5, 0x0, {hw}, Not Active, Not Active, {power_cap}"


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _Proc()
    s.lines = lines
    return s


def test_only_samples_inside_the_timed_region_count():
    now = time.perf_counter()  # the region began 0.2 s ago and ends at stop()
    s = _sampler([(now - 2.0, _line(900, hw="Active")),   # warm-up, before the region
                  (now - 0.19, _line(2070)), (now - 0.14, _line(2055)), (now - 0.09, _line(2070)),
                  (now + 5.0, _line(1000, hw="Active"))])  # long after the region
    s.w0 = now - 0.2
    c = s.stop()
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == []


def test_throttle_reasons_inside_the_region_are_reported():
    now = time.perf_counter()
    s = _sampler([(now + 0.01, _line(1800, hw="Active")), (now + 0.02, _line(2070, power_cap="Active")),
                  (now + 0.03, "garbled line")])
    s.w0 = now
    c = s.stop()
    assert c["samples"] == 2
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert c["sm_mhz"] == (1800.0 + 2070.0) / 2


def test_no_sampler_process():
    s = bench.ClockSampler(0)
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
