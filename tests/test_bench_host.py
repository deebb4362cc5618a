"""CPU checks of the benchmark's host logic: the scope table's algorithmic
bytes behind the roofline line, and the clock record taken during the timed
region (median SM clock, throttle reasons seen)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_projection_bytes_follow_the_scope_table():
    # templates once, the 24 skinning transforms (48 B) of every visible
    # instance, one 40-byte record per splat
    st = {"instances_visible": 3119, "splats": 22705852}
    assert bench.project_scope_bytes(st, 231_000_000) == 231_000_000 + 3119 * 24 * 48 + 22705852 * 40


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _Thread:
    def join(self, timeout=None):
        pass


def _sampled(lines):
    c = bench.ClockSampler(0)
    c.proc, c.t, c.lines = _Proc(), _Thread(), list(lines)
    return c.stop()


def test_clock_record_takes_the_median_and_every_active_reason():
    row = "0, {sm}, 2070, 1100.5, 0x0, {hw}, Not Active, Not Active, {cap}"
    rec = _sampled([row.format(sm=2070, hw="Not Active", cap="Not Active"),
                    row.format(sm=1980, hw="Not Active", cap="Active"),
                    row.format(sm=2070, hw="Active", cap="Not Active"),
                    "garbage line", ""])
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"],
                   "samples": 3}


def test_clock_record_is_absent_without_samples():
    assert _sampled([]) is None
    assert bench.ClockSampler(0).stop() is None  # nvidia-smi never started
