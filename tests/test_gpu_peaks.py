"""The library's arithmetic-pipe microbenchmarks (mhd_measure_pipe_peaks):
finite positive rates, ordered as the hardware's units are (FP64 FMA well
below FP32 FMA, the BF16 tensor MMA above FP32 FMA), and none above the
nominal rate of its unit by more than the clock can explain."""
import math

import pytest

pytestmark = pytest.mark.gpu

# 152 SMs x 2.07 GHz x lanes x 2 flops: FP64 2 lanes, FP32 128 lanes per SM
NOMINAL = {"fp64_fma_tflops": 152 * 2.07 * 2 * 2 / 1e3, "fp32_fma_tflops": 152 * 2.07 * 128 * 2 / 1e3}


def test_pipe_peaks():
    import torch
    from paper_2606_12753_gb300 import mhd
    s = torch.cuda.Stream()
    p = mhd.mhd_measure_pipe_peaks(s.cuda_stream)
    for k in ("fp64_fma_tflops", "fp32_fma_tflops", "bf16_mma_sync_tflops"):
        assert math.isfinite(p[k]) and p[k] > 0, (k, p)
    assert p["fp64_fma_tflops"] < 0.1 * p["fp32_fma_tflops"], p
    assert p["bf16_mma_sync_tflops"] > p["fp32_fma_tflops"], p
    for k, nom in NOMINAL.items():
        assert p[k] < 1.05 * nom, (k, p[k], nom)
    assert all(t > 0 for t in p["ms"])
