"""Timed CPU runs of the oracle for the benchmark's CPU-baseline leg.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.  These are process-pool workers: each builds the
config-2 aquifer from its seed and times the oracle on a bounded sample, so
that the benchmark can report what the FP64 CPU method achieves on the host.
"""
from __future__ import annotations

import time

import numpy as np

from . import contour, direct, fgmres_sh, fv


def shift_sample(args):
    """O1 (contour + SuperLU) on `count` config-2 shifted systems of one time.
    args = (seed, time index, first node, count); returns (count, seconds)."""
    seed, t_index, k0, count = args
    import workloads as W
    prob = W.config2(seed=seed)
    K, m = fv.assemble(prob)
    z, _ = contour.nodes_weights(prob.times[t_index % len(prob.times)], prob.Nz)
    b = fv.rhs(prob, len(prob.src_cells) // 2)
    t0 = time.perf_counter()
    for k in range(k0, k0 + count):
        direct.shifted_solve(K, m, z[k % len(z)], b / z[k % len(z)])
    return count, time.perf_counter() - t0


def fgmres_group(args):
    """The paper's own configuration: Algorithm 1 (FGMRES-Sh) with exact LU preconditioners and
    the tau_bar1 / tau_bar2 3:2 schedule (Sec. 3), for one source and one time group of config 2.
    args = (seed, source, group, groups, tol); returns (shifts, converged, iterations, seconds)."""
    seed, source, group, groups, tol = args
    import workloads as W
    prob = W.config2(seed=seed)
    K, m = fv.assemble(prob)
    order = np.argsort(prob.times)
    tg = np.array_split(order, groups)[group]
    zs = np.concatenate([contour.nodes_weights(prob.times[t], prob.Nz)[0] for t in tg])
    taus = contour.tau_schedule(zs, "flexible", 400)
    b = fv.rhs(prob, source)
    t0 = time.perf_counter()
    _, nit, conv = fgmres_sh.solve(K, m, b, zs, taus, tol=tol, maxit=400)
    return len(zs), int(np.sum(conv >= 0)), nit, time.perf_counter() - t0
