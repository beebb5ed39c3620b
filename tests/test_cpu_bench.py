"""Host-side arithmetic of bench.py's reported rates.

The network timing leg (`bench.py --only unet`) reports TFLOP/s from a MAC count per full-size
pixel.  That count is pinned here to the convolutions the CPU oracle of the same network
actually executes: every conv2d call of `oracle.unet.forward` is counted as
(output elements) x (input channels) x 9 on a small image."""
import numpy as np
import pytest
import torch

import bench
from oracle import unet as U


def test_unet_mac_count_matches_the_oracle_network():
    calls = []
    real = torch.nn.functional.conv2d

    def counting(x, w, b=None, *a, **k):
        y = real(x, w, b, *a, **k)
        calls.append((int(x.shape[1]), int(w.shape[0]), int(y.numel()) * int(x.shape[1]) * int(w.shape[2] * w.shape[3])))
        return y

    H, W = 32, 48
    theta = torch.zeros(U.num_params(), dtype=torch.float64)
    x = torch.zeros(1, H, W, 5, dtype=torch.float64)
    torch.nn.functional.conv2d = counting
    try:
        U.forward(theta, x)
    finally:
        torch.nn.functional.conv2d = real
    assert [(ci, co) for ci, co, _ in calls] == [(ci, co) for ci, co, _ in bench.UNET_CONVS]
    macs = sum(m for _, _, m in calls)
    assert macs / (H * W) == pytest.approx(bench.UNET_MAC_PER_PIXEL, rel=0, abs=1e-9)
    assert bench.UNET_MAC_PER_PIXEL == 30816


def test_vcycle_roofline_bytes_and_flops():
    # (16 + 16 + 24 / R) x 4/3 bytes per fine cell per V-cycle, R right-hand sides share the coefficients
    assert bench.vcycle_bytes_per_unit(27) == pytest.approx(43.85185185185185)
    assert bench.vcycle_bytes_per_unit(1) == pytest.approx(56.0 * 4.0 / 3.0)
    # (24 (pre + post) + 28 + 18) x 4/3 FP32 flops per fine cell per V-cycle
    assert bench.inner_flops_per_unit(0, 2) == pytest.approx(94.0 * 4.0 / 3.0)
    assert bench.inner_flops_per_unit(2, 2) == pytest.approx(142.0 * 4.0 / 3.0)
    assert np.isfinite(bench.vcycle_bytes_per_unit(0))
