"""The FP32 FMA microbenchmark that gives the raster kernels' roofline its denominator
(`gs_measure_fp32_peak`, scalar and packed-pair FMA chains): its rate must be physically
possible, at most what 128 FMA lanes per SM can do at the GPU's maximum SM clock (2 FLOPs
per FMA; a rate above that would mean the chains were optimised away), and not far below it
(a rate under half of it would mean the kernel is not filling the SMs)."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_fp32_peak_is_physical():
    import torch
    from paper_2603_09632_gb300 import _lib as L
    import bench
    dev = torch.device("cuda", 0)
    try:
        max_mhz = bench.NvmlClockSampler(dev).max_mhz
    except OSError:
        pytest.skip("NVML not available for the maximum SM clock")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lanes_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    tf, ms = L.gs_measure_fp32_peak(8192)
    assert ms > 0.0
    assert 0.5 * lanes_tflops < tf <= 1.02 * lanes_tflops, (tf, lanes_tflops)
