"""The machine-ceiling probes on the GPU: the special-function exponential rate
and random 8-byte gather rates from buffers that fit L1/L2 and that do not."""
import pytest

from paper_1810_00188_gb300 import mcrt

pytestmark = pytest.mark.gpu


def test_ex2_probe_rate_and_clock_are_plausible():
    import torch
    per_s, mhz = mcrt.mcrt_probe_ex2(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 < mhz < 3000.0
    per_clk_sm = per_s / (sms * mhz * 1e6)
    # a special-function unit: a few to a few tens of results per clock per SM
    assert 2.0 < per_clk_sm < 64.0, per_clk_sm


def test_gather_probe_orders_cache_levels():
    small = mcrt.mcrt_probe_gather(0, 2 << 20)    # the 64^3 FP32 field: L1/L2 resident
    large = mcrt.mcrt_probe_gather(0, 4 << 30)    # far beyond L2: HBM sectors
    assert small > 0 and large > 0
    assert small > large
    # a random 8-byte load from HBM moves at least one 32-byte sector, so the
    # useful rate stays well under the copy bandwidth (nominal 7.9 TB/s)
    assert 8.0 * large < 8e12 / 2
