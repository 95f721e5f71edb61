"""The FP32 FMA-throughput probe used for the compute roof of the roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_1111_2142_gb300 import lwacm as lw
    props = torch.cuda.get_device_properties(0)
    tf, ms = lw.measure_fp32_peak(2048)
    # 128 FP32 lanes per SM, 2 flops per FMA, at most ~2.1 GHz
    ceiling = props.multi_processor_count * 128 * 2 * 2.1e9 / 1e12
    print(f"FP32 FMA rate {tf:.1f} TFLOP/s ({ms:.2f} ms); ceiling at 2.1 GHz {ceiling:.1f}")
    assert ms > 0
    assert 0.25 * ceiling < tf < 1.05 * ceiling
