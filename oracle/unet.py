"""CPU oracle of the learned-preconditioner network (test infrastructure).

The same U-Net as the CUDA implementation, written with plain PyTorch CPU
ops in float64: 3x3 convolutions (padding 1), 2x2 average pooling, nearest
2x up-sampling, channel concatenation [up-sampled, skip], ReLU, and a mean
squared error over the two output channels.  Parameters use the library's
flat layout: for each layer W[9][cout][cin] (tap = 3 ky + kx) then b[cout].
Gradients come from autograd; pinned by finite differences in
tests/test_oracle_unet.py.
"""
from __future__ import annotations

import numpy as np
import torch

# (cin, cout, relu) per layer; input channels 5 padded to 16, output 2 padded to 16
LAYERS = [(16, 16, 1), (16, 16, 1), (16, 32, 1), (32, 32, 1), (32, 32, 1), (32, 32, 1), (32, 64, 1), (64, 64, 1),
          (96, 32, 1), (32, 32, 1), (64, 32, 1), (32, 32, 1), (48, 16, 1), (16, 16, 1), (16, 16, 0)]
IN_CHANNELS = 5
OUT_CHANNELS = 2


def num_params():
    return sum(9 * ci * co + co for ci, co, _ in LAYERS)


def unpack(theta):
    out, off = [], 0
    for ci, co, _ in LAYERS:
        W = theta[off:off + 9 * co * ci].reshape(9, co, ci)
        off += 9 * co * ci
        b = theta[off:off + co]
        off += co
        out.append((W, b))
    return out


def _conv(x, W, b, relu):
    # x: [n, C, H, W]; W[tap][co][ci] with tap = 3 ky + kx -> conv2d weight [co, ci, 3, 3]
    w = W.reshape(3, 3, W.shape[1], W.shape[2]).permute(2, 3, 0, 1)
    y = torch.nn.functional.conv2d(x, w, b, padding=1)
    return torch.relu(y) if relu else y


def forward(theta, x):
    """theta: float64 tensor [P]; x: float64 tensor [n, H, W, 5] -> output [n, H, W, 2]."""
    P = unpack(theta)
    n, H, W_, _ = x.shape
    h = torch.zeros(n, 16, H, W_, dtype=x.dtype)
    h[:, :IN_CHANNELS] = x.permute(0, 3, 1, 2)
    pool = lambda t: torch.nn.functional.avg_pool2d(t, 2)
    up = lambda t: t.repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)
    c = lambda i, t: _conv(t, P[i][0], P[i][1], LAYERS[i][2])
    s0 = c(1, c(0, h))
    s1 = c(3, c(2, pool(s0)))
    s2 = c(5, c(4, pool(s1)))
    bb = c(7, c(6, pool(s2)))
    d2 = c(9, c(8, torch.cat([up(bb), s2], 1)))
    d1 = c(11, c(10, torch.cat([up(d2), s1], 1)))
    d0 = c(13, c(12, torch.cat([up(d1), s0], 1)))
    out = c(14, d0)
    return out[:, :OUT_CHANNELS].permute(0, 2, 3, 1)


def loss_and_grad(theta_np, x_np, target_np):
    theta = torch.tensor(theta_np, dtype=torch.float64, requires_grad=True)
    x = torch.tensor(x_np, dtype=torch.float64)
    t = torch.tensor(target_np, dtype=torch.float64)
    out = forward(theta, x)
    loss = ((out - t) ** 2).mean()
    loss.backward()
    return float(loss), theta.grad.numpy().copy(), out.detach().numpy()
