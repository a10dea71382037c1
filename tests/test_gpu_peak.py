"""The FMA-loop microbenchmark that gives the ALU rooflines their denominator:
its FP32 figure must sit near the nominal 148 SMs x 128 lanes x 2 FLOP x clock
(a loop the compiler had removed would read far above it), and FP64 must be
positive and below FP32."""
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts deselect these
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402


def test_fma_peak_is_plausible():
    f32 = ocf.fma_peak(False)
    f64 = ocf.fma_peak(True)
    nominal = 148 * 128 * 2 * 2.032e9 / 1e12      # 77 TFLOP/s at the maximum SM clock
    assert 0.5 * nominal <= f32 <= 1.05 * nominal, f32
    assert 0.0 < f64 < f32, (f64, f32)
