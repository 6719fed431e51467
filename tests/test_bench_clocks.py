"""The bench's clock check (host logic): which timed regions are measured
again.  A hardware or thermal slowdown, or SM clocks well below their maximum
with no reason given, rejects a region; a power cap alone does not."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def clocks(sm, mx, reasons, samples=5):
    return {"sm_mhz": sm, "sm_max_mhz": mx, "reasons": reasons, "samples": samples}


def test_clean_and_power_capped_regions_are_kept():
    assert not bench.clocks_rejected(clocks(2070.0, 2070.0, []))
    assert not bench.clocks_rejected(clocks(1950.0, 2070.0, ["sw_power_cap"]))
    assert not bench.clocks_rejected(clocks(1500.0, 2070.0, ["sw_power_cap"]))


def test_slowdowns_and_clock_locks_are_rejected():
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(clocks(2070.0, 2070.0, [r]))
        assert bench.clocks_rejected(clocks(1800.0, 2070.0, ["sw_power_cap", r]))
    assert bench.clocks_rejected(clocks(1500.0, 2070.0, []))      # well below max, no reason: a lock


def test_no_samples_is_not_a_rejection():
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(clocks(None, None, [], samples=0))


class _FakeTimer(bench.Timer):
    def __init__(self, records):
        super().__init__(None, None, 1, 0)
        self.records, self.calls = list(records), 0

    def run(self, fn, steps, warmup, sample_clocks=False):
        self.calls += 1
        return {"total_ms": 1.0, "per_ms": [1.0], "wall_s": 0.1, "clocks": self.records.pop(0)}


def test_run_checked_measures_once_more_only_when_rejected():
    t = _FakeTimer([clocks(2070.0, 2070.0, [])])
    assert t.run_checked(None, 1, 1)["clocks"]["sm_mhz"] == 2070.0 and t.calls == 1
    t = _FakeTimer([clocks(2070.0, 2070.0, ["hw_slowdown"]), clocks(2070.0, 2070.0, [])])
    r = t.run_checked(None, 1, 1)
    assert t.calls == 2 and r["clocks"]["reasons"] == [] and r["clocks"]["remeasured_after"]["reasons"] == ["hw_slowdown"]
