"""Solve the forward (and adjoint) problems of several independent aquifers together.

`forward_batch(engines, times)` calls lt_forward_batch: each Engine keeps its
own grid, wells and options; the library interleaves their outer iterations
on per-context streams so the GPU runs the aquifers concurrently.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Sequence

import numpy as np

from . import _lib as L
from .engine import LtError


def forward_batch(engines: Sequence, times_list: Sequence, allow_unconverged: bool = False):
    """Return (list of h[ns][nr][nt] numpy arrays, list of stats dicts)."""
    n = len(engines)
    if n == 0:
        return [], []
    lib = engines[0].lib
    ts = [np.ascontiguousarray(np.asarray(t, dtype=np.float64)) for t in times_list]
    hs = [np.zeros((e.ns, e.nr, t.size)) for e, t in zip(engines, ts)]
    ctxs = (C.c_void_p * n)(*[e.h.value for e in engines])
    nts = (C.c_int * n)(*[t.size for t in ts])
    tptr = (C.c_void_p * n)(*[t.ctypes.data for t in ts])
    hptr = (C.c_void_p * n)(*[h.ctypes.data for h in hs])
    stats = (L.LtStats * n)()
    rc = lib.lt_forward_batch(n, ctxs, nts, tptr, hptr, 0, stats)
    if rc != L.LT_OK and not (allow_unconverged and rc == L.LT_ERR_NOT_CONVERGED):
        msgs = "; ".join(lib.lt_last_error(e.h).decode() for e in engines if lib.lt_last_error(e.h))
        raise LtError(rc, f"lt_forward_batch: {lib.lt_strerror(rc).decode()}: {msgs}")
    return hs, [stats[i].as_dict() for i in range(n)]


def adjoint_batch(engines: Sequence, times_list: Sequence, J=None, g=None, grad=None, h=None,
                  allow_unconverged: bool = False):
    """Adjoint Jacobians (J: list of CUDA float64 [ns][nr][nt][2][ncell], entries may be None) or
    vector-Jacobian products (g: list of CUDA float64 [ns][nr][nt] -> grad: list of CUDA float64
    [2][ncell]) of several aquifers through lt_adjoint_batch; h: optional list of CUDA float64
    [ns][nr][nt] for the measurements.  Returns the list of stats dicts."""
    n = len(engines)
    if n == 0:
        return []
    lib = engines[0].lib
    ts = [np.ascontiguousarray(np.asarray(t, dtype=np.float64)) for t in times_list]

    def ptrs(lst):
        if lst is None:
            return None
        return (C.c_void_p * n)(*[(x.data_ptr() if x is not None else 0) for x in lst])

    ctxs = (C.c_void_p * n)(*[e.h.value for e in engines])
    nts = (C.c_int * n)(*[t.size for t in ts])
    tptr = (C.c_void_p * n)(*[t.ctypes.data for t in ts])
    stats = (L.LtStats * n)()
    rc = lib.lt_adjoint_batch(n, ctxs, nts, tptr, ptrs(J), ptrs(g), ptrs(grad), ptrs(h), stats)
    if rc != L.LT_OK and not (allow_unconverged and rc == L.LT_ERR_NOT_CONVERGED):
        msgs = "; ".join(lib.lt_last_error(e.h).decode() for e in engines if lib.lt_last_error(e.h))
        raise LtError(rc, f"lt_adjoint_batch: {lib.lt_strerror(rc).decode()}: {msgs}")
    return [stats[i].as_dict() for i in range(n)]
