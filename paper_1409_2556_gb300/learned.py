"""Learned initial guess for the preconditioner solves: network handle,
training-pair generation with the library's own multigrid, and training.

Everything numerical runs in liblt.so (tensor-core U-Net kernels, Adam,
multigrid, the contour nodes, the network's input channels and targets);
this module draws synthetic residuals, moves tensors and drives the loop.
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

    def set_wait_polls(self, polls: int):
        """Poll limit of the convolutions' bounded waits (0: every wait runs out at once)."""
        self._check(self.lib.lt_unet_set_wait_polls(self.h, int(polls)), "set_wait_polls")

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
    """e = multigrid solve of (K + tau_i M) e_i = r_i (r: CUDA complex64 [n, ncell] viewed as float32 pairs)."""
    import torch
    t = _tau_array(tau)
    e = torch.zeros_like(r)
    rc = engine.lib.lt_precond_apply(engine.h, len(t), t.ctypes.data_as(C.c_void_p), C.c_void_p(r.data_ptr()),
                                     C.c_void_p(e.data_ptr()), int(cycles))
    engine._check(rc, "lt_precond_apply")
    return e


def _tau_array(tau):
    return np.ascontiguousarray(np.asarray([[complex(v).real, complex(v).imag] for v in tau], dtype=np.float64))


def contour_nodes(t: float, Nz: int, project: bool = True):
    """Talbot nodes of time t from the library (upper half, Re projected to >= 0 if asked)."""
    lib = L.load()
    z = np.zeros((Nz // 2, 2))
    rc = lib.lt_contour_nodes(float(t), int(Nz), int(project), z.ctypes.data_as(C.c_void_p), None)
    if rc != 0:
        raise LtError(rc, f"lt_contour_nodes(t={t}, Nz={Nz})")
    return z[:, 0] + 1j * z[:, 1]


def sample_shifts(rng, n: int, Nz: int = 32, t_range=(10.0, 1e4)):
    """Preconditioner-style shifts: a random Talbot node of a random time, Re projected to >= 0."""
    t = np.exp(rng.uniform(np.log(t_range[0]), np.log(t_range[1]), n))
    k = rng.integers(0, Nz // 2, n)
    return np.array([contour_nodes(ti, Nz)[ki] for ti, ki in zip(t, k)])


def pairs_from_residuals(engine: Engine, tau, r, cycles: int = 40):
    """Network inputs [n, ncell, 5] and targets [n, ncell, 2] for residuals r (CUDA complex64
    [n, ncell]) and shifts tau: the library solves (K + tau M) e = r by multigrid and forms the
    channels and the unit-RMS target D e on the device (lt_learned_pairs)."""
    import torch
    n = r.shape[0]
    N = r.shape[1]
    t = _tau_array(tau)
    rr = torch.view_as_real(r).contiguous()
    x = torch.empty((n, N, IN_CHANNELS), dtype=torch.float32, device=r.device)
    y = torch.empty((n, N, 2), dtype=torch.float32, device=r.device)
    rc = engine.lib.lt_learned_pairs(engine.h, n, t.ctypes.data_as(C.c_void_p), C.c_void_p(rr.data_ptr()),
                                     int(cycles), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()))
    engine._check(rc, "lt_learned_pairs")
    return x, y


def krylov_residuals(engine: Engine, max_n: int):
    """The Krylov vectors v_j (and their shifts tau_j) of the engine's last solve: the residuals the
    preconditioner actually receives inside Algorithm 1 (lt_krylov_vectors)."""
    import torch
    r = torch.zeros((max_n, engine.ncell), dtype=torch.complex64, device=f"cuda:{engine.device}")
    tau = np.zeros((max_n, 2))
    n = C.c_int()
    rr = torch.view_as_real(r)
    engine._check(engine.lib.lt_krylov_vectors(engine.h, max_n, C.c_void_p(rr.data_ptr()),
                                               tau.ctypes.data_as(C.c_void_p), C.byref(n)), "lt_krylov_vectors")
    k = n.value
    return r[:k].contiguous(), tau[:k, 0] + 1j * tau[:k, 1]


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


def make_pairs(engine: Engine, prob, n: int, rng, cycles: int = 40, batch: int = 256, krylov: bool = True):
    """(input, target) pairs on the engine's grid, reshaped to [n, ny, nx, C].  With krylov=True
    the residuals are the Krylov vectors of a forward solve of `prob` on this engine (the vectors
    the preconditioner solves inside Algorithm 1), topped up with synthetic residuals if the solve
    produced fewer than n; else all residuals are synthetic (point sources, smooth fields, noise)."""
    import torch
    dev = torch.device("cuda", engine.device)
    rs, taus = [], []
    if krylov:
        engine.set_sources(prob.src_cells, prob.Q)
        engine.set_receivers(prob.rec_cells)
        engine.set_options(Nz=prob.Nz, tol=prob.tol, groups=prob.groups)
        engine.forward(prob.times, allow_unconverged=True)
        r, tau = krylov_residuals(engine, n)
        rs.append(r)
        taus.append(tau)
    have = sum(x.shape[0] for x in rs)
    if have < n:
        rs.append(random_residuals(rng, n - have, prob.ny, prob.nx, dev))
        taus.append(sample_shifts(rng, n - have))
    r = torch.cat(rs)
    tau = np.concatenate(taus)
    xs, ys = [], []
    for i0 in range(0, n, batch):
        k = min(batch, n - i0)
        x, y = pairs_from_residuals(engine, tau[i0:i0 + k], r[i0:i0 + k].contiguous(), cycles)
        xs.append(x.reshape(k, prob.ny, prob.nx, IN_CHANNELS))
        ys.append(y.reshape(k, prob.ny, prob.nx, 2))
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
