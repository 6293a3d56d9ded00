"""The micro-benchmark kernels behind the rooflines' denominators: every
kind launches, and the measured rates sit between a floor no B300 falls
below and the nominal unit counts at the maximum clock (148 SMs, 2032 MHz:
128 FP32 lanes, 16 MUFU lanes per SM) with 10 % slack."""
import pytest
import torch

import bench

pytestmark = pytest.mark.gpu


def test_peak_rates_are_plausible():
    dev = torch.device("cuda", 0)
    p = bench.measure_peaks(torch, dev, 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ghz = 2.032
    assert 0.3 * sms * 256 * ghz / 1e3 < p["fp32_tflops"] <= 1.1 * sms * 256 * ghz / 1e3
    assert 0.0 < p["fp64_tflops"] < p["fp32_tflops"]
    assert 0.0 < p["mufu_tanh_gops"] <= 1.1 * sms * 32 * ghz
    assert 0.0 < p["mufu_ex2_gops"] <= 1.1 * sms * 32 * ghz
    assert p["graph_node_per_s"] > p["launch_per_s"] > 1e3
