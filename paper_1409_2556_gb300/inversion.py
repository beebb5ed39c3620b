"""Quasi-linear geostatistical inversion (Sec. 5.1, Algorithm 2) driven through the C ABI.

Each iteration is one lt_geostat_step call (Jacobian, FFT covariance product, FP64 GEMM,
Cholesky solve and update, all in the library's kernels); this module only sets the grid to the
new estimate and loops.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .engine import Engine


def geostat_step(eng: Engine, times, y, R, sigma2: float, ell: float, allow_unconverged: bool = False):
    """One iteration at the engine's current kappa: returns (s_next, beta, xi, h)."""
    t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
    yy = np.ascontiguousarray(np.asarray(y, dtype=np.float64).ravel())
    rr = np.ascontiguousarray(np.asarray(R, dtype=np.float64).ravel())
    s_next = np.zeros(eng.ncell)
    beta = np.zeros(1)
    xi = np.zeros(yy.size)
    h = np.zeros(yy.size)
    st = L.LtStats()
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = eng.lib.lt_geostat_step(eng.h, t.size, p(t), p(yy), p(rr), float(sigma2), float(ell), p(s_next), p(beta),
                                 p(xi), p(h), C.byref(st))
    eng.last_stats = st.as_dict()
    eng._check(rc, "lt_geostat_step", (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ())
    return s_next, float(beta[0]), xi, h


def gauss_newton(eng: Engine, prob, y, R, sigma2: float, ell: float, s0, iters: int = 10, tol: float = 1e-10):
    """Algorithm 2 from s0 on the engine (grid shape, wells and options of `prob`); returns (s, history)."""
    s = np.asarray(s0, dtype=np.float64).copy()
    hist = []
    for _ in range(iters):
        eng.setup_grid(np.exp(s).reshape(prob.kappa.shape), prob.Ss, prob.dx, prob.dy, prob.dz, prob.bc,
                       getattr(prob, "Sy", None))
        eng.set_sources(prob.src_cells, prob.Q)
        eng.set_receivers(prob.rec_cells)
        s_new, beta, xi, h = geostat_step(eng, prob.times, y, R, sigma2, ell)
        step = float(np.linalg.norm(s_new - s) / max(np.linalg.norm(s_new), 1e-300))
        hist.append(dict(step=step, beta=beta, misfit=float(np.sum((np.ravel(y) - h) ** 2 / np.ravel(R)))))
        s = s_new
        if step < tol:
            break
    return s, hist
