"""Python front end of the engine: one `Engine` per GPU context.

Thin wrapper over the C ABI (include/lt.h): it converts numpy arrays and
torch tensors to pointers and raises on non-OK status codes.  Device buffers
come from PyTorch (memory and streams only); all arithmetic runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _lib as L


class LtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Engine:
    """Laplace-transform forward/adjoint engine on one CUDA device."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = L.load()
        h = C.c_void_p()
        rc = self.lib.lt_create(C.byref(h), int(device))
        if rc != L.LT_OK:
            raise LtError(rc, f"lt_create(device={device}) failed: {self.lib.lt_strerror(rc).decode()}")
        self.h = h
        self.device = device
        self.opts = L.LtOpts()
        self.lib.lt_default_options(C.byref(self.opts))
        self.last_stats = None
        self.ns = self.nr = 0
        self.ncell = 0
        if stream is not None:
            self.set_stream(stream)

    # -------------------------------------------------------------- plumbing
    def _check(self, rc: int, what: str, allow=()):
        if rc == L.LT_OK or rc in allow:
            return rc
        msg = self.lib.lt_last_error(self.h).decode()
        raise LtError(rc, f"{what}: {self.lib.lt_strerror(rc).decode()}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.lt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (legacy default)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.lt_set_stream(self.h, C.c_void_p(handle or 0)), "lt_set_stream")

    # -------------------------------------------------------------- problem
    def setup_grid(self, kappa, Ss, dx: float, dy: float, dz: float, bc: Sequence[int] = (0, 0, 0, 0, 1, 1),
                   Sy=None):
        k = _f64(kappa)
        s = _f64(Ss)
        if k.ndim == 2:
            k = k[None]
            s = s[None]
        nz, ny, nx = k.shape
        if s.shape != k.shape:
            raise ValueError("kappa and Ss shapes differ")
        b = np.ascontiguousarray(np.asarray(bc, dtype=np.int32))
        if b.size != 6:
            raise ValueError("bc needs 6 face codes")
        sy = None if Sy is None else _f64(Sy).ravel()
        if sy is not None and sy.size != k.size:
            raise ValueError("Sy needs one value per cell")
        self._check(self.lib.lt_setup_grid(self.h, nx, ny, nz, float(dx), float(dy), float(dz), _ptr(k), _ptr(s),
                                           _ptr(b), _ptr(sy) if sy is not None else None), "lt_setup_grid")
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz

    def set_sources(self, cells, Q):
        c = _i64(cells)
        q = _f64(Q)
        self._check(self.lib.lt_set_sources(self.h, c.size, _ptr(c), _ptr(q)), "lt_set_sources")
        self.ns = c.size

    def set_source_rates(self, terms):
        """terms: per source (amplitudes, decay rates) of q_s(t) = sum_j a_j exp(-lambda_j t);
        None restores the constant rates."""
        if terms is None:
            self._check(self.lib.lt_set_source_rates(self.h, 0, None, None, None), "lt_set_source_rates")
            return
        n = np.ascontiguousarray([len(np.atleast_1d(a)) for a, _ in terms], dtype=np.int32)
        a = _f64(np.concatenate([np.atleast_1d(a) for a, _ in terms]))
        lam = _f64(np.concatenate([np.atleast_1d(l) for _, l in terms]))
        self._check(self.lib.lt_set_source_rates(self.h, len(terms), _ptr(n), _ptr(a), _ptr(lam)),
                    "lt_set_source_rates")

    def set_initial_state(self, phi0):
        """phi0: float64 [ncell] initial head, or None for phi(0) = 0."""
        if phi0 is None:
            self._check(self.lib.lt_set_initial_state(self.h, None), "lt_set_initial_state")
            return
        p = _f64(phi0).ravel()
        if p.size != self.ncell:
            raise ValueError(f"phi0 needs {self.ncell} entries")
        self._check(self.lib.lt_set_initial_state(self.h, _ptr(p)), "lt_set_initial_state")

    def set_receivers(self, cells):
        c = _i64(cells)
        self._check(self.lib.lt_set_receivers(self.h, c.size, _ptr(c)), "lt_set_receivers")
        self.nr = c.size

    def set_options(self, **kw):
        o = L.LtOpts()
        C.memmove(C.byref(o), C.byref(self.opts), C.sizeof(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        self._check(self.lib.lt_set_options(self.h, C.byref(o)), "lt_set_options")
        self.opts = o

    def load_problem(self, prob, **opts):
        """Configure from a workloads.Problem (grid, wells, Nz, tol, groups)."""
        self.setup_grid(prob.kappa, prob.Ss, prob.dx, prob.dy, prob.dz, prob.bc, getattr(prob, "Sy", None))
        self.set_sources(prob.src_cells, prob.Q)
        self.set_receivers(prob.rec_cells)
        if getattr(prob, "rate_terms", None) is not None:
            self.set_source_rates(prob.rate_terms)
        if getattr(prob, "phi0", None) is not None:
            self.set_initial_state(prob.phi0)
        o = dict(Nz=prob.Nz, tol=prob.tol, groups=prob.groups)
        o.update(opts)
        self.set_options(**o)

    # -------------------------------------------------------------- solves
    def forward(self, times, out=None, allow_unconverged: bool = False):
        """h[ns][nr][nt]; `out` may be a CUDA torch tensor (float64, contiguous) or None (numpy result)."""
        t = _f64(times)
        st = L.LtStats()
        allow = (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        if out is None:
            h = np.zeros((self.ns, self.nr, t.size))
            rc = self.lib.lt_forward(self.h, t.size, _ptr(t), _ptr(h), 0, C.byref(st))
            res = h
        else:
            _check_dev(out, (self.ns, self.nr, t.size))
            rc = self.lib.lt_forward(self.h, t.size, _ptr(t), C.c_void_p(out.data_ptr()), 1, C.byref(st))
            res = out
        self.last_stats = st.as_dict()
        self._check(rc, "lt_forward", allow)
        return res

    def forward_noalloc(self, times, out, allow_unconverged: bool = False):
        """Same as forward() into a CUDA float64 tensor `out` [ns][nr][nt], without any
        device allocation by the library (its buffers come from a fixed static region;
        for callers whose device memory is owned by their own pool allocator, or who
        cannot afford the device synchronisation of cudaMalloc/cudaFree).  Calls that
        overlap on the GPU share that region and race."""
        t = _f64(times)
        _check_dev(out, (self.ns, self.nr, t.size))
        st = L.LtStats()
        rc = self.lib.lt_forward_noalloc(self.h, t.size, _ptr(t), C.c_void_p(out.data_ptr()), C.byref(st))
        self.last_stats = st.as_dict()
        self._check(rc, "lt_forward_noalloc", (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return out

    def crank_nicolson(self, times, steps: int, out=None, allow_unconverged: bool = False):
        """h[ns][nr][nt] by Crank-Nicolson time stepping on the GPU (lt_crank_nicolson)."""
        t = _f64(times)
        st = L.LtStats()
        allow = (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        if out is None:
            h = np.zeros((self.ns, self.nr, t.size))
            rc = self.lib.lt_crank_nicolson(self.h, t.size, _ptr(t), int(steps), _ptr(h), 0, C.byref(st))
            res = h
        else:
            _check_dev(out, (self.ns, self.nr, t.size))
            rc = self.lib.lt_crank_nicolson(self.h, t.size, _ptr(t), int(steps), C.c_void_p(out.data_ptr()), 1,
                                            C.byref(st))
            res = out
        self.last_stats = st.as_dict()
        self._check(rc, "lt_crank_nicolson", allow)
        return res

    def forward_fields(self, times, out=None, allow_unconverged: bool = False):
        t = _f64(times)
        st = L.LtStats()
        allow = (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        if out is None:
            phi = np.zeros((self.ns, t.size, self.ncell))
            rc = self.lib.lt_forward_fields(self.h, t.size, _ptr(t), _ptr(phi), 0, C.byref(st))
            res = phi
        else:
            _check_dev(out, (self.ns, t.size, self.ncell))
            rc = self.lib.lt_forward_fields(self.h, t.size, _ptr(t), C.c_void_p(out.data_ptr()), 1, C.byref(st))
            res = out
        self.last_stats = st.as_dict()
        self._check(rc, "lt_forward_fields", allow)
        return res

    def adjoint_jacobian(self, times, J, allow_unconverged: bool = False):
        """J: CUDA float64 tensor [ns][nr][nt][2][ncell] (filled in place)."""
        t = _f64(times)
        _check_dev(J, (self.ns, self.nr, t.size, 2, self.ncell))
        st = L.LtStats()
        rc = self.lib.lt_adjoint_jacobian(self.h, t.size, _ptr(t), C.c_void_p(J.data_ptr()), C.byref(st))
        self.last_stats = st.as_dict()
        self._check(rc, "lt_adjoint_jacobian", (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return J

    def adjoint_vjp(self, times, g, grad, h=None, allow_unconverged: bool = False):
        """g: CUDA float64 [ns][nr][nt]; grad: CUDA float64 [2][ncell]; h: optional CUDA [ns][nr][nt]."""
        t = _f64(times)
        _check_dev(g, (self.ns, self.nr, t.size))
        _check_dev(grad, (2, self.ncell))
        if h is not None:
            _check_dev(h, (self.ns, self.nr, t.size))
        st = L.LtStats()
        rc = self.lib.lt_adjoint_vjp(self.h, t.size, _ptr(t), C.c_void_p(g.data_ptr()), C.c_void_p(grad.data_ptr()),
                                     C.c_void_p(h.data_ptr() if h is not None else 0), 1, C.byref(st))
        self.last_stats = st.as_dict()
        self._check(rc, "lt_adjoint_vjp", (L.LT_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return grad


def _check_dev(t, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
