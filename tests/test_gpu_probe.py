"""lat_probe_rates: the measured integer-pipe rates that serve as roofline
denominators.  Each must be positive and no higher than the pipe's width
allows at the device's maximum clock (a rate above that would mean the
microkernel's work was optimised away), and the full Philox4x32-10 block
rate must be of the order the widening-multiply rate allows (a block is
twenty widening multiplies, 40 IMAD-ops; the slack covers the two chain
layouts' different operand patterns)."""
import pytest

from paper_2502_18624_gb300 import binding as b

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible(gpu):
    import torch
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_hz = 2.2e9                       # above the GB300's 2.07 GHz maximum SM clock
    r = b.lat_probe_rates()
    assert all(t > 0 for t in r["seconds"])
    # lanes per SM and clock: 64 logic lanes, 16 population-count lanes, 64 IMAD lanes
    assert 0 < r["lop3_per_s"] <= sms * 64 * max_hz
    assert 0 < r["popc_per_s"] <= sms * 16 * max_hz
    assert 0 < r["imad32_per_s"] <= sms * 64 * max_hz
    assert 0 < r["imad_ops_per_s"] <= sms * 64 * max_hz
    assert 0 < r["philox_blocks_per_s"] <= r["imad_ops_per_s"] / 40 * 1.5
    # the rates are not wildly below the pipes either (a broken timing would be)
    assert r["lop3_per_s"] > 0.3 * sms * 64 * 1.0e9
    assert r["popc_per_s"] > 0.3 * sms * 16 * 1.0e9
