"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds only input generation: grids, Gaussian random fields for
log-conductivity and log-storage, well locations and output times.  It holds
none of the method's arithmetic (no operator assembly, no contour, no
solver), so that both sides of a parity test can draw identical inputs
without sharing any computation.

The paper's experiments (Sec. 4.1) use a 100 m square domain, a mean
transmissivity of 1e-4 m^2/s, storativity 1e-5, and a random log-field with
an exponential covariance kernel; its own fields are not available, so the
fields here are seeded samples with that structure.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

L_DOMAIN = 100.0          # m, side of the square domain (Sec. 4.1)
Q_RATE = 8.5e-4           # m^3/s, 0.85 L/s pumping rate (Sec. 4.1)
KAPPA_MEAN = 1e-4         # m/s (2D: m^2/s transmissivity), Sec. 4.1
SS_CONST = 1e-5           # 1/m (2D: storativity), Sec. 4.1

# boundary codes per face (x-, x+, y-, y+, z-, z+)
BC_DIRICHLET = 0
BC_NEUMANN = 1
BC_WATERTABLE = 2        # linearised water table (no flux; storage S_y per unit face area)


@dataclass
class Problem:
    """One aquifer: grid, coefficients, wells and output times."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    kappa: np.ndarray            # [nz][ny][nx] float64, > 0
    Ss: np.ndarray               # [nz][ny][nx] float64, > 0
    bc: Tuple[int, ...]          # 6 face codes
    src_cells: np.ndarray        # int64 [ns]
    Q: np.ndarray                # float64 [ns]
    rec_cells: np.ndarray        # int64 [nr]
    times: np.ndarray            # float64 [nt]
    Nz: int                      # contour nodes (full contour; Nz/2 shifts solved)
    tol: float
    groups: int = 1              # preconditioner-shift groups over the times
    phi0: Optional[np.ndarray] = None   # [ncell] float64 initial head (None: phi(0) = 0)
    Sy: Optional[np.ndarray] = None     # [ncell] float64 specific yield, used on water-table faces
    # per source: (amplitudes a_j [m^3/s], decay rates lambda_j >= 0 [1/s]) of the rate
    # q_s(t) = sum_j a_j exp(-lambda_j t); None: the constant rate Q_s switched on at t = 0
    rate_terms: Optional[List[Tuple[np.ndarray, np.ndarray]]] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz


def cell_index(i: int, j: int, k: int, nx: int, ny: int) -> int:
    """Linear cell index, x fastest: (k*ny + j)*nx + i."""
    return (k * ny + j) * nx + i


def gaussian_field(shape: Tuple[int, ...], variance: float, corr_len: Tuple[float, ...],
                   seed: int) -> np.ndarray:
    """Zero-mean stationary Gaussian field with exponential covariance
    C(r) = variance * exp(-r), r = || (d_i / corr_len_i) ||_2 in cells.

    Sampled by circulant embedding on a torus padded to twice each extent;
    negative embedding eigenvalues are clipped to zero (the sample is then
    very slightly off the exact covariance, which does not matter for a
    synthetic input).  Returns float64 of the given shape (C order).
    """
    rng = np.random.default_rng(seed)
    pshape = tuple(2 * s for s in shape)
    axes = []
    for s, ps, lc in zip(shape, pshape, corr_len):
        d = np.arange(ps, dtype=np.float64)
        d = np.minimum(d, ps - d)          # torus distance
        axes.append(d / max(lc, 1e-30))
    grids = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    cov = variance * np.exp(-r)
    lam = np.fft.fftn(cov).real
    lam = np.clip(lam, 0.0, None)
    xi = rng.standard_normal(pshape) + 1j * rng.standard_normal(pshape)
    f = np.fft.fftn(np.sqrt(lam / np.prod(pshape)) * xi)
    sl = tuple(slice(0, s) for s in shape)
    return np.ascontiguousarray(f.real[sl])


def log_times(t0: float, t1: float, n: int) -> np.ndarray:
    return np.geomspace(t0, t1, n)


def _lattice(n: int, k: int) -> List[int]:
    return [int(round(v)) for v in np.linspace(0.2 * n, 0.8 * n, k)]


def config1(n: int = 64, Nz: int = 16, tol: float = 1e-10) -> Problem:
    """64x64 homogeneous 2D box, Dirichlet all round, one central source,
    four observation cells 8 cells from the source, 8 log-spaced times in
    [10, 1e4] s, single preconditioner shift."""
    h = L_DOMAIN / n
    kappa = np.full((1, n, n), KAPPA_MEAN)
    Ss = np.full((1, n, n), SS_CONST)
    c = n // 2
    src = np.array([cell_index(c, c, 0, n, n)], dtype=np.int64)
    d = min(8, max(1, n // 8))
    rec = np.array([cell_index(c + d, c, 0, n, n), cell_index(c - d, c, 0, n, n),
                    cell_index(c, c + d, 0, n, n), cell_index(c, c - d, 0, n, n)], dtype=np.int64)
    return Problem(n, n, 1, h, h, 1.0, kappa, Ss,
                   (BC_DIRICHLET,) * 4 + (BC_NEUMANN,) * 2,
                   src, np.full(1, Q_RATE), rec, log_times(10.0, 1e4, 8), Nz, tol,
                   groups=1, name=f"homogeneous-{n}x{n}")


def config2(n: int = 256, Nz: int = 32, tol: float = 1e-8, seed: int = 2,
            variance: float = 1.5, corr: float = 20.0, nt: int = 12, groups: int = 3,
            n_src_side: int = 3, n_rec_side: int = 5) -> Problem:
    """Heterogeneous 2D aquifer: log-kappa Gaussian field (exponential
    covariance), constant Ss, a 3x3 lattice of pumping wells, a 5x5 lattice
    of observation wells, 12 log-spaced times in [10, 1e4] s."""
    h = L_DOMAIN / n
    logk = np.log(KAPPA_MEAN) + gaussian_field((n, n), variance, (corr, corr), seed)
    kappa = np.exp(logk)[None]
    Ss = np.full((1, n, n), SS_CONST)
    if n_src_side == 3:
        sl = [n // 4, n // 2, 3 * n // 4]
    else:
        sl = _lattice(n, n_src_side)
    src = np.array([cell_index(i, j, 0, n, n) for j in sl for i in sl], dtype=np.int64)
    rl = _lattice(n, n_rec_side)
    rec = np.array([cell_index(i, j, 0, n, n) for j in rl for i in rl], dtype=np.int64)
    return Problem(n, n, 1, h, h, 1.0, kappa, Ss,
                   (BC_DIRICHLET,) * 4 + (BC_NEUMANN,) * 2,
                   src, np.full(len(src), Q_RATE), rec, log_times(10.0, 1e4, nt), Nz, tol,
                   groups=groups, name=f"lognormal-{n}x{n}-var{variance}")


def config3(nxy: int = 128, nz: int = 32, Nz: int = 16, tol: float = 1e-8,
            seeds: Tuple[int, int] = (3, 4), nt: int = 10, n_src_side: int = 4,
            n_rec_side: int = 4, rec_layers: Optional[List[int]] = None) -> Problem:
    """3D aquifer with log-normal kappa (variance 1.0, correlation 16x16x4
    cells) and log-normal Ss (variance 0.25), Dirichlet lateral faces,
    no-flow top and bottom; 16 sources on the mid layer, 48 receivers on
    three layers."""
    h = L_DOMAIN / nxy
    logk = np.log(KAPPA_MEAN) + gaussian_field((nz, nxy, nxy), 1.0, (4.0 * nz / 32, 16.0 * nxy / 128, 16.0 * nxy / 128), seeds[0])
    logs = np.log(SS_CONST) + gaussian_field((nz, nxy, nxy), 0.25, (4.0 * nz / 32, 16.0 * nxy / 128, 16.0 * nxy / 128), seeds[1])
    kappa = np.exp(logk)
    Ss = np.exp(logs)
    sl = _lattice(nxy, n_src_side)
    zm = nz // 2
    src = np.array([cell_index(i, j, zm, nxy, nxy) for j in sl for i in sl], dtype=np.int64)
    if rec_layers is None:
        rec_layers = [nz // 4, nz // 2, (3 * nz) // 4]
    rl = [v + max(1, nxy // 16) for v in _lattice(nxy, n_rec_side)]
    rl = [min(v, nxy - 1) for v in rl]
    rec = np.array([cell_index(i, j, k, nxy, nxy) for k in rec_layers for j in rl for i in rl], dtype=np.int64)
    return Problem(nxy, nxy, nz, h, h, h, kappa, Ss,
                   (BC_DIRICHLET,) * 4 + (BC_NEUMANN,) * 2,
                   src, np.full(len(src), Q_RATE), rec, log_times(10.0, 1e4, nt), Nz, tol,
                   groups=1, name=f"3d-{nxy}x{nxy}x{nz}")


def config5_aquifers(seed: int = 5, count: int = 40) -> List[Problem]:
    """Uneven batch of independent 2D aquifers: side from {96,...,384},
    log-kappa variance in [0.5, 3.0], 4-16 sources, 16-64 receivers, 8 times,
    24 contour nodes."""
    rng = np.random.default_rng(seed)
    out = []
    for a in range(count):
        n = int(rng.choice([96, 128, 192, 256, 384]))
        var = float(rng.uniform(0.5, 3.0))
        ns = int(rng.integers(4, 17))
        nr = int(rng.integers(16, 65))
        h = L_DOMAIN / n
        logk = np.log(KAPPA_MEAN) + gaussian_field((n, n), var, (20.0, 20.0), seed * 1000 + a)
        cells = rng.choice(np.arange(n * n), size=ns + nr, replace=False)
        out.append(Problem(n, n, 1, h, h, 1.0, np.exp(logk)[None], np.full((1, n, n), SS_CONST),
                           (BC_DIRICHLET,) * 4 + (BC_NEUMANN,) * 2,
                           np.sort(cells[:ns]).astype(np.int64), np.full(ns, Q_RATE),
                           np.sort(cells[ns:]).astype(np.int64), log_times(10.0, 1e4, 8), 24, 1e-8,
                           groups=2, name=f"aquifer{a}-{n}-var{var:.2f}"))
    return out


def random_problem(nx: int, ny: int, nz: int = 1, variance: float = 1.0, seed: int = 0,
                   ns: int = 2, nr: int = 3, nt: int = 3, Nz: int = 16, tol: float = 1e-10,
                   bc: Optional[Tuple[int, ...]] = None, ss_variance: float = 0.0,
                   groups: int = 1, t_range: Tuple[float, float] = (10.0, 1e4)) -> Problem:
    """Small seeded heterogeneous problem of arbitrary shape (tests)."""
    rng = np.random.default_rng(seed + 7919)
    L = L_DOMAIN
    dx = L / nx
    dy = L / ny
    dz = 1.0 if nz == 1 else dx
    shape = (nz, ny, nx)
    corr = (max(1.0, nz / 4), max(1.0, ny / 6), max(1.0, nx / 6))
    logk = np.log(KAPPA_MEAN) + (gaussian_field(shape, variance, corr, seed) if variance > 0 else 0.0)
    logs = np.log(SS_CONST) + (gaussian_field(shape, ss_variance, corr, seed + 1) if ss_variance > 0 else 0.0)
    kappa = np.ascontiguousarray(np.broadcast_to(np.exp(logk), shape)).astype(np.float64)
    Ss = np.ascontiguousarray(np.broadcast_to(np.exp(logs), shape)).astype(np.float64)
    if bc is None:
        bc = (BC_DIRICHLET,) * 4 + (BC_NEUMANN,) * 2
    cells = rng.choice(np.arange(nx * ny * nz), size=ns + nr, replace=False)
    times = np.geomspace(t_range[0], t_range[1], nt) if nt > 1 else np.array([np.sqrt(t_range[0] * t_range[1])])
    return Problem(nx, ny, nz, dx, dy, dz, kappa, Ss, tuple(bc),
                   cells[:ns].astype(np.int64), rng.uniform(0.5, 1.5, ns) * Q_RATE,
                   cells[ns:].astype(np.int64), times, Nz, tol, groups=groups,
                   name=f"random-{nx}x{ny}x{nz}")


def with_initial_state_and_rates(prob: Problem, seed: int = 0, phi0_amp: float = 0.05,
                                 n_terms: int = 3, rates: bool = True, initial: bool = True) -> Problem:
    """The same aquifer with a non-zero initial head and time-varying pumping rates.

    phi0: a smooth seeded Gaussian field (correlation a quarter of the grid) scaled to an RMS of
    `phi0_amp` m.  Rates: per source, its constant rate Q_s plus n_terms - 1 decaying terms
    a_j exp(-lambda_j t) with |a_j| <= Q_s and 1/lambda_j log-uniform in [30, 3000] s (within the
    output times), so that q_s(t) stays positive."""
    import copy
    rng = np.random.default_rng(seed + 104729)
    out = copy.copy(prob)
    if initial:
        shape = (prob.nz, prob.ny, prob.nx)
        corr = tuple(max(1.0, s / 4.0) for s in shape)
        f = gaussian_field(shape, 1.0, corr, seed + 17).ravel()
        out.phi0 = np.ascontiguousarray(phi0_amp * f / max(np.sqrt(np.mean(f * f)), 1e-300))
    if rates:
        terms = []
        for s in range(len(prob.src_cells)):
            a = [float(prob.Q[s])]
            lam = [0.0]
            for _ in range(n_terms - 1):
                a.append(float(rng.uniform(-0.4, 0.8)) * float(prob.Q[s]))
                lam.append(1.0 / float(np.exp(rng.uniform(np.log(30.0), np.log(3000.0)))))
            terms.append((np.array(a), np.array(lam)))
        out.rate_terms = terms
    out.name = prob.name + ("-phi0" if initial else "") + ("-rates" if rates else "")
    return out


def with_water_table(prob: Problem, face: int = 5, sy: float = 0.2, seed: int = 0,
                     variance: float = 0.0) -> Problem:
    """The same aquifer with a linearised water table on one face (default z+, the top):
    specific yield sy (times a log-normal factor of the given variance, seeded) per cell."""
    import copy
    out = copy.copy(prob)
    bc = list(prob.bc)
    bc[face] = BC_WATERTABLE
    out.bc = tuple(bc)
    f = np.ones(prob.ncell)
    if variance > 0:
        shape = (prob.nz, prob.ny, prob.nx)
        corr = tuple(max(1.0, s / 4.0) for s in shape)
        f = np.exp(gaussian_field(shape, variance, corr, seed + 29).ravel())
    out.Sy = np.ascontiguousarray(sy * f)
    out.name = prob.name + "-watertable"
    return out
