"""The measured FP32 FMA issue rate behind the traversal kernels' "alu"
roofline: within the range the SM count and clock allow."""
import pytest

from paper_2501_02747_gb300 import ivm

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    ctx = ivm.Context(0, torch.cuda.current_stream(0))
    try:
        rate = ivm.ivm_fp32_peak(ctx)
    finally:
        ctx.close()
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2.2e9   # lanes x a clock above any boost
    assert 0.2 * nominal < rate < nominal, (rate, nominal)
