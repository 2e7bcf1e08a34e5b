"""The measured FMA throughput that bench.py reports the stage kernels'
arithmetic against: positive, below the nominal lane-count roof (152 SMs x
128 FP32 / 2 FP64 FMA lanes x 2 FLOP at the 2070 MHz maximum clock, with 10 %
slack for clock reporting), and FP32 far above FP64 on GB300."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_fma_peaks():
    import torch
    from paper_2207_04252_gb300 import build
    build.build()
    from paper_2207_04252_gb300 import rossbi as R
    torch.cuda.init()
    f32 = R.rossbi_measure_fma_peak(False)
    f64 = R.rossbi_measure_fma_peak(True)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print(f"FMA peaks: FP32 {f32 / 1e12:.2f} TFLOP/s, FP64 {f64 / 1e12:.3f} TFLOP/s on {sms} SMs")
    assert math.isfinite(f32) and math.isfinite(f64) and f32 > 0 and f64 > 0
    assert f32 <= 1.1 * sms * 128 * 2 * 2070e6
    assert f32 > 10 * f64
