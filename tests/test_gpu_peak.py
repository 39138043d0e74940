"""The FP32 throughput probe behind the ALU roofline: packed f32x2 and scalar FMA loops
on every SM.  A GB300 has 152 SMs of 128 FP32 lanes at about 2 GHz (78 TFLOP/s scalar at
2 flops per lane and clock); the probe must land near that, and the packed form must
not fall below the scalar one."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    from paper_2510_13866_gb300 import fp32_peak

    scalar = fp32_peak(0, packed=False)
    packed = fp32_peak(0, packed=True)
    print(f"\nFP32 FMA: scalar {scalar:.1f} TFLOP/s, packed f32x2 {packed:.1f} TFLOP/s")
    assert 30.0 < scalar < 100.0
    assert 0.9 * scalar < packed < 220.0


def test_fp64_peak_is_plausible():
    """GB300's FP64 rate is a small fraction of its FP32 rate (about 1.2 TFLOP/s dense)."""
    from paper_2510_13866_gb300 import fp32_peak, fp64_peak

    dp = fp64_peak(0)
    print(f"\nFP64 FMA: {dp:.2f} TFLOP/s")
    assert 0.2 < dp < 0.5 * fp32_peak(0, packed=False)
