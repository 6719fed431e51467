"""The measurement probes run on the GPU and give rates that agree with the
work they time: the FP64 FMA rate lies between a quarter of and the unit-count
ceiling (SMs x 2 FMA per clock x 2 flop x the highest SM clock), and the random
read rate out of an L2-sized buffer is at least that out of a 2 GB buffer."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probe(lib):
    """GB300's FP64 unit count is two fused multiply-adds per SM and clock; the
    probe's rate, divided by the SM clock it read during the launch, lands
    just under it."""
    import torch
    r = lib.spmv_probe_fp64(3)
    assert r["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 500 < r["sm_mhz"] < 2500, r
    assert 1.7 < r["fma_per_clock_per_sm"] <= 2.02, r
    assert r["ms"] > 0.5


def test_gather_probe_l2_vs_dram(lib):
    l2 = lib.spmv_probe_gather(6_201_600, 3)
    dram = lib.spmv_probe_gather(1 << 28, 2)
    assert l2["gathers_per_s"] > 1e10 and dram["gathers_per_s"] > 1e9 and 500 < l2["sm_mhz"] < 2500
    assert l2["gathers_per_s"] >= 0.95 * dram["gathers_per_s"], (l2, dram)
