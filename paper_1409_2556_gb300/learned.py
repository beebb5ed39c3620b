"""Learned initial guess for the preconditioner solves: network handle,
training-pair generation with the library's own multigrid, and training.

Everything numerical runs in liblt.so (tensor-core U-Net kernels, Adam,
multigrid); this module prepares tensors and drives the loop.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Tuple

import numpy as np

from . import _lib as L
from .engine import Engine, LtError

IN_CHANNELS = 5


class UNet:
    def __init__(self, device: int = 0, seed: int = 0):
        self.lib = L.load()
        h = C.c_void_p()
        rc = self.lib.lt_unet_create(C.byref(h), int(device), int(seed))
        if rc != 0:
            raise LtError(rc, "lt_unet_create failed")
        self.h = h
        self.device = device
        self.nparams = self.lib.lt_unet_num_params(h)

    def _check(self, rc, what):
        if rc != 0:
            raise LtError(rc, f"{what}: {self.lib.lt_unet_last_error(self.h).decode()}")

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        self._check(self.lib.lt_unet_get_params(self.h, out.ctypes.data_as(C.c_void_p), self.nparams), "get_params")
        return out

    def set_params(self, theta):
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        self._check(self.lib.lt_unet_set_params(self.h, t.ctypes.data_as(C.c_void_p), t.size), "set_params")

    def forward(self, x):
        """x: CUDA float32 tensor [n, H, W, 5] -> CUDA float32 [n, H, W, 2]."""
        import torch
        n, H, W, c = x.shape
        out = torch.empty((n, H, W, 2), dtype=torch.float32, device=x.device)
        self._check(self.lib.lt_unet_forward(self.h, n, H, W, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr())),
                    "forward")
        return out

    def grad(self, x, target) -> Tuple[float, np.ndarray]:
        n, H, W, _ = x.shape
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = C.c_double()
        self._check(self.lib.lt_unet_grad(self.h, n, H, W, C.c_void_p(x.data_ptr()), C.c_void_p(target.data_ptr()),
                                          g.ctypes.data_as(C.c_void_p), C.byref(loss)), "grad")
        return loss.value, g

    def train_step(self, x, target, lr: float) -> float:
        n, H, W, _ = x.shape
        loss = C.c_double()
        self._check(self.lib.lt_unet_train_step(self.h, n, H, W, C.c_void_p(x.data_ptr()),
                                                C.c_void_p(target.data_ptr()), C.c_float(lr), C.byref(loss)),
                    "train_step")
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lt_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def precond_apply(engine: Engine, tau, r, cycles: int):
    """e = multigrid solve of (K + tau_i M) e_i = r_i (r: CUDA complex64 [n, ncell])."""
    import torch
    t = np.ascontiguousarray(np.asarray([[complex(v).real, complex(v).imag] for v in tau], dtype=np.float64))
    e = torch.zeros_like(r)
    rc = engine.lib.lt_precond_apply(engine.h, len(t), t.ctypes.data_as(C.c_void_p), C.c_void_p(r.data_ptr()),
                                     C.c_void_p(e.data_ptr()), int(cycles))
    engine._check(rc, "lt_precond_apply")
    return e


def features(prob, r, tau):
    """Network input [n, ny, nx, 5] and per-image scale s for residuals r (complex [n, ncell]) of
    shifts tau (n values): Re r/s, Im r/s, normalised log kappa, Re(tau) m/D, Im(tau) m/D."""
    import torch
    n = r.shape[0]
    ny, nx = prob.ny, prob.nx
    dev = r.device
    s = torch.sqrt(torch.mean(torch.abs(r) ** 2, dim=1)).clamp_min(1e-30)
    lk = np.log(prob.kappa[0])
    lk = (lk - lk.mean()) / max(lk.std(), 1e-12)
    D, m = operator_diag(prob)
    x = torch.zeros((n, ny, nx, IN_CHANNELS), dtype=torch.float32, device=dev)
    rr = (r / s[:, None]).reshape(n, ny, nx)
    x[..., 0] = rr.real
    x[..., 1] = rr.imag
    x[..., 2] = torch.tensor(lk, dtype=torch.float32, device=dev)[None]
    ratio = torch.tensor((m / D).reshape(ny, nx), dtype=torch.float32, device=dev)
    tau_t = torch.tensor(np.asarray(tau, dtype=np.complex128), device=dev)
    x[..., 3] = tau_t.real.float()[:, None, None] * ratio[None]
    x[..., 4] = tau_t.imag.float()[:, None, None] * ratio[None]
    return x, s


def operator_diag(prob):
    """Diagonal D (sum of face transmissibilities incl. Dirichlet) and m of the 2D FV operator."""
    k = prob.kappa[0]
    ny, nx = k.shape
    ax, ay = prob.dy * prob.dz / prob.dx, prob.dx * prob.dz / prob.dy
    harm = lambda a, b: 2 * a * b / (a + b)
    D = np.zeros((ny, nx))
    tx = ax * harm(k[:, :-1], k[:, 1:])
    ty = ay * harm(k[:-1, :], k[1:, :])
    D[:, :-1] += tx; D[:, 1:] += tx; D[:-1, :] += ty; D[1:, :] += ty
    bc = prob.bc
    if bc[0] == 0: D[:, 0] += 2 * k[:, 0] * ax
    if bc[1] == 0: D[:, -1] += 2 * k[:, -1] * ax
    if bc[2] == 0: D[0, :] += 2 * k[0, :] * ay
    if bc[3] == 0: D[-1, :] += 2 * k[-1, :] * ay
    m = prob.Ss[0] * prob.dx * prob.dy * prob.dz
    return D.ravel(), m.ravel()


# modified Talbot contour (Sec. 2.2): shifts of the training pairs are drawn from it
_SIGMA, _MU, _ALPHA, _NU = -0.6122, 0.5017, 0.6407, 0.2645


def sample_shifts(rng, n: int, Nz: int = 32, t_range=(10.0, 1e4)):
    """Preconditioner-style shifts: a Talbot node of a random time, Re projected to >= 0."""
    t = np.exp(rng.uniform(np.log(t_range[0]), np.log(t_range[1]), n))
    th = rng.uniform(0.05, np.pi - 0.05, n)
    z = (Nz / t) * (_SIGMA + _MU * th / np.tan(_ALPHA * th) + 1j * _NU * th)
    return np.maximum(z.real, 0.0) + 1j * z.imag


def random_residuals(rng, n: int, ny: int, nx: int, device):
    """Mixture of point sources, smooth random fields and white noise (complex float32 [n, ny*nx])."""
    import torch
    r = np.zeros((n, ny, nx), dtype=np.complex128)
    for i in range(n):
        kind = i % 3
        if kind == 0:
            r[i, rng.integers(ny), rng.integers(nx)] = np.exp(1j * rng.uniform(0, 2 * np.pi))
        elif kind == 1:
            w = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
            ky = np.fft.fftfreq(ny)[:, None]
            kx = np.fft.fftfreq(nx)[None, :]
            ell = rng.uniform(0.02, 0.3)
            r[i] = np.fft.ifft2(np.fft.fft2(w) * np.exp(-(kx ** 2 + ky ** 2) / (2 * ell ** 2)))
        else:
            r[i] = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
        r[i] /= np.sqrt(np.mean(np.abs(r[i]) ** 2))
    return torch.tensor(r.reshape(n, ny * nx), dtype=torch.complex64, device=device)


def make_pairs(engine: Engine, prob, n: int, rng, cycles: int = 40, batch: int = 256):
    """(input features, target) pairs on the engine's grid: residuals r, shifts tau,
    targets D e normalised to unit RMS, e the multigrid solution of (K + tau M) e = r
    (the solver rescales the network's direction by a minimal-residual coefficient)."""
    import torch
    dev = torch.device("cuda", engine.device)
    D, _ = operator_diag(prob)
    Dt = torch.tensor(D, dtype=torch.float32, device=dev)
    xs, ys = [], []
    for i0 in range(0, n, batch):
        k = min(batch, n - i0)
        tau = sample_shifts(rng, k)
        r = random_residuals(rng, k, prob.ny, prob.nx, dev)
        e = precond_apply(engine, tau, torch.view_as_real(r).contiguous(), cycles)
        e = torch.view_as_complex(e)
        x, s = features(prob, r, tau)
        de = e * Dt[None]
        nrm = torch.sqrt(torch.mean(torch.abs(de) ** 2, dim=1)).clamp_min(1e-30)
        tgt = (de / nrm[:, None].to(torch.complex64)).reshape(k, prob.ny, prob.nx)
        ys.append(torch.stack([tgt.real, tgt.imag], -1).float().contiguous())
        xs.append(x)
    return torch.cat(xs), torch.cat(ys)


def training_fields(seeds=range(8), n: int = 64, variance: float = 1.5):
    """Config-1-style 64x64 aquifers with log-normal kappa (training set)."""
    import workloads as W
    return [W.config2(n=n, seed=100 + s, variance=variance, corr=20.0 * n / 256.0, nt=4, groups=1) for s in seeds]


def train(net: UNet, pairs, steps: int = 1500, batch: int = 32, lr: float = 1e-3, rng=None, log_every: int = 0):
    """Adam on random mini-batches of the pairs; returns the loss history."""
    import torch
    rng = rng or np.random.default_rng(0)
    x, y = pairs
    hist = []
    for it in range(steps):
        idx = torch.tensor(rng.choice(x.shape[0], size=batch, replace=False), device=x.device)
        xb = x.index_select(0, idx).contiguous()
        yb = y.index_select(0, idx).contiguous()
        l = net.train_step(xb, yb, lr * (0.3 if it > 0.7 * steps else 1.0))
        hist.append(l)
        if log_every and it % log_every == 0:
            print(f"step {it} loss {l:.4e}", flush=True)
    return hist
