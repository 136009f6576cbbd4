"""Measured on-chip peaks (sp_measure_peaks): the denominators of the region
kernel's shared-memory and FP32 roofline lines.  Checked against the SM count
and clock of the device: conflict-free 16-byte reads deliver at most 128
bytes per clock per SM and FP32 FMAs at most 128 per clock per SM (256
flops), and a healthy device reaches a good part of both."""
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import sp  # noqa: E402

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_within_the_hardware_bounds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    smem_gbs, fp32_tflops = sp.sp_measure_peaks(torch.cuda.current_stream().cuda_stream)
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_ghz = 2.2  # above any SM clock of the part
    assert 0.3 * sms * 128 * 1.0 < smem_gbs < sms * 128 * max_ghz, smem_gbs
    assert 0.3 * sms * 256 * 1.0 / 1e3 < fp32_tflops < sms * 256 * max_ghz / 1e3, fp32_tflops
    print(f"\nshared memory {smem_gbs:.0f} GB/s, FP32 {fp32_tflops:.1f} TFLOP/s on {sms} SMs")
