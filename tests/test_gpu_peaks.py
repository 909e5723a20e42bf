"""The roofline denominators measured by rp_measure_peaks on the GPU: each rate is positive and
within what the hardware can do -- FP32 FMA between half and 110 % of the lanes' peak at the
maximum SM clock (152 SMs x 128 lanes x 2 flops x clock), FP64 below the FP32 rate, and the L2
read bandwidth above the HBM copy bandwidth (the buffer is L2-resident) and below 100 TB/s."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp

    pk = rp.measure_peaks()
    props = torch.cuda.get_device_properties(0)
    lanes_peak = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    print("measured peaks:", pk)
    assert 0.5 * lanes_peak <= pk["fp32_tflops"] <= 1.1 * lanes_peak
    assert 0.0 < pk["fp64_tflops"] < pk["fp32_tflops"]
    assert 6000.0 < pk["l2_gbs"] < 100000.0
    assert min(pk["fp32_ms"], pk["fp64_ms"], pk["l2_ms"]) > 0.5
