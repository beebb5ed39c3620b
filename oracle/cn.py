"""O3: Crank-Nicolson time stepping of M phi' + K phi = sum_s q_s(t) e_s,
phi(0) = phi_0 (the time-stepping method the paper compares against,
Sec. 1 and Sec. 5.3).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

    (M + dt/2 K) phi^{n+1} = (M - dt/2 K) phi^n + dt/2 (b(t_n) + b(t_{n+1}))

The step source at t = 0 (and a rough initial state) excites the stiff modes
that Crank-Nicolson does not damp, so the first interval starts with four
backward-Euler quarter steps (Rannacher start); each interval between
consecutive output times is then covered by uniform steps, and Richardson
extrapolation over two step sizes (error O(dt^2)) gives the result.  An
independent cross-check of O1; not the parity reference.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fv, source


def _march(K, m, qb, phi0, times, steps_per_interval):
    """qb(t): the source vector at time t."""
    M = sp.diags(m)
    phi = phi0.copy()
    out = []
    t_prev = 0.0
    cache = {}
    for ti, t in enumerate(times):
        span = t - t_prev
        nsteps = steps_per_interval
        dt = span / nsteps
        tc = t_prev
        if ti == 0:
            # Rannacher start: 4 backward-Euler steps of dt/4 cover the first dt
            be = spla.splu((M + (dt / 4) * K).tocsc())
            for _ in range(4):
                tc += dt / 4
                phi = be.solve(m * phi + (dt / 4) * qb(tc))
            nsteps -= 1
        key = round(dt, 15)
        if key not in cache:
            cache[key] = spla.splu((M + (dt / 2) * K).tocsc())
        lu = cache[key]
        Bm = (M - (dt / 2) * K).tocsr()
        for _ in range(nsteps):
            phi = lu.solve(Bm @ phi + (dt / 2) * (qb(tc) + qb(tc + dt)))
            tc += dt
        out.append(phi.copy())
        t_prev = t
    return np.array(out)


def heads(prob, steps_per_interval: int = 400, extrapolate: bool = True):
    """h[ns][nr][nt] by Crank-Nicolson (+ Richardson)."""
    K, m = fv.assemble(prob)
    phi0 = source.initial_state(prob)
    h = np.zeros((len(prob.src_cells), len(prob.rec_cells), len(prob.times)))
    for s in range(len(prob.src_cells)):
        e = np.zeros(prob.ncell)
        e[prob.src_cells[s]] = 1.0
        qb = lambda t, e=e, s=s: source.q_time(prob, s, t) * e
        p1 = _march(K, m, qb, phi0, prob.times, steps_per_interval)
        if extrapolate:
            p2 = _march(K, m, qb, phi0, prob.times, 2 * steps_per_interval)
            p = (4.0 * p2 - p1) / 3.0
        else:
            p = p1
        h[s] = p[:, prob.rec_cells].T
    return h
