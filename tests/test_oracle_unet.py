"""Pins for the network oracle: autograd gradient vs central finite differences."""
import numpy as np

from oracle import unet


def test_param_count_and_fd_gradient():
    rng = np.random.default_rng(0)
    P = unet.num_params()
    assert P == sum(9 * a * b + b for a, b, _ in unet.LAYERS)
    theta = rng.standard_normal(P) * 0.1
    x = rng.standard_normal((2, 16, 16, 5))
    t = rng.standard_normal((2, 16, 16, 2))
    loss, g, _ = unet.loss_and_grad(theta, x, t)
    idx = rng.choice(P, 12, replace=False)
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (unet.loss_and_grad(tp, x, t)[0] - unet.loss_and_grad(tm, x, t)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
