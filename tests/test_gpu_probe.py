"""rb_fma_rate: the measured FMA rate that serves as the denominator of the FP64 outer
residual's arithmetic roofline.  The figures are checked for what the hardware fixes: both
rates are positive, finite and below the issue limit of 152 SMs x 128 FP32 lanes x 2 flops at
2.1 GHz (about 82 TFLOP/s), and on this part FP64 is far slower than FP32."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_06363_gb300 import rb  # noqa: E402


def test_fma_rates_are_plausible():
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9
    r32 = rb.fma_rate(False)
    r64 = rb.fma_rate(True)
    for r in (r32, r64):
        assert math.isfinite(r) and 0.0 < r <= ceiling
    assert r64 < r32
    assert r32 > 0.25 * ceiling   # the probe keeps every FP32 lane busy most of the time
