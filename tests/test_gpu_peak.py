"""The measured FP32 lane rate (af_fp32_lane_rate), the rooflines' denominator: a
plain FMA loop reaches most of, and not more than, SMs x 128 lanes x the maximum
SM clock."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402


def test_fp32_lane_rate_is_near_the_nominal_lane_count():
    props = torch.cuda.get_device_properties(0)
    rate = af.fp32_lane_rate()
    nominal = props.multi_processor_count * 128 * 2032e6
    print(f"FP32 lane rate {rate / 1e12:.2f} T lane-op/s, {rate / nominal:.3f} of "
          f"{props.multi_processor_count} SMs x 128 x 2032 MHz")
    assert 0.5 * nominal < rate < 1.1 * nominal
