"""Measurements as a differentiable function of (log kappa, log Ss).

`LaplaceMeasurements.apply(log_kappa, log_Ss, engine, problem)` returns
h[s][r][t] (float64, on the engine's device).  Its backward is the
Laplace-domain adjoint of Sec. 5.2, evaluated by lt_adjoint_vjp (receiver
solves plus the fused sensitivity assembly); no Jacobian is materialised.
Both directions run in the library's CUDA kernels; PyTorch only carries the
tensors.
"""
from __future__ import annotations

import numpy as np
import torch


class LaplaceMeasurements(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_kappa: torch.Tensor, log_Ss: torch.Tensor, engine, problem):
        kap = torch.exp(log_kappa.detach()).to(torch.float64).cpu().numpy()
        ss = torch.exp(log_Ss.detach()).to(torch.float64).cpu().numpy()
        engine.setup_grid(kap, ss, problem.dx, problem.dy, problem.dz, problem.bc)
        engine.set_sources(problem.src_cells, problem.Q)
        engine.set_receivers(problem.rec_cells)
        dev = torch.device("cuda", engine.device)
        h = torch.zeros((len(problem.src_cells), len(problem.rec_cells), len(problem.times)), dtype=torch.float64,
                        device=dev)
        engine.forward(problem.times, out=h)
        torch.cuda.synchronize(dev)
        ctx.engine = engine
        ctx.problem = problem
        ctx.shape = tuple(log_kappa.shape)
        ctx.devices = (log_kappa.device, log_Ss.device)
        return h

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        eng, prob = ctx.engine, ctx.problem
        dev = torch.device("cuda", eng.device)
        gd = g.detach().to(device=dev, dtype=torch.float64).contiguous()
        grad = torch.zeros((2, int(np.prod(ctx.shape))), dtype=torch.float64, device=dev)
        eng.adjoint_vjp(prob.times, gd, grad)
        torch.cuda.synchronize(dev)
        gk = grad[0].reshape(ctx.shape).to(ctx.devices[0])
        gs = grad[1].reshape(ctx.shape).to(ctx.devices[1])
        return gk, gs, None, None


def measurements(log_kappa, log_Ss, engine, problem):
    return LaplaceMeasurements.apply(log_kappa, log_Ss, engine, problem)
