"""Measured FMA throughput used as the ALU roofline denominator (GPU only)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05143_gb300 import measure_fma_peak
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32 = measure_fma_peak("fp32")
    fp64 = measure_fma_peak("fp64")
    # 128 FP32 lanes per SM, two flops per FMA, clock between 0.8 and 2.2 GHz
    assert sms * 128 * 2 * 0.8e9 * 0.7 < fp32 < sms * 128 * 2 * 2.2e9 * 1.05
    assert 0 < fp64 < fp32
