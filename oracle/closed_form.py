"""O2: eigenfunction expansion of the semi-discrete FV system for a
homogeneous box (exact for M phi' + K phi = q(t) e_s, phi(0) = phi_0; Sec. 2.1).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

Per axis with n cells, the 1D FV operator (unit transmissibility) has
  Dirichlet both ends (ghost half a cell away, boundary diagonal 3):
      v_p(j) ~ sin(p pi (j + 1/2) / n),  lam_p = 4 sin^2(p pi / 2n), p = 1..n
  Neumann both ends:
      v_p(j) ~ cos(p pi (j + 1/2) / n),  lam_p = 4 sin^2(p pi / 2n), p = 0..n-1
(j 0-based, columns normalised to unit length).  With T_x = kappa A_x / dx etc. and M = Ss V I, K separates:
  K = kappa (A_x/dx L_x (x) I (x) I + ...),  eigenvalues kappa sum_d (A_d / d_d) lam_{p_d},
so each mode (mu = K-eigenvalue / (Ss V)) obeys a_p' + mu a_p = v_p(s) q(t) / (Ss V),
a_p(0) = v_p . phi_0, and for q(t) = sum_j c_j e^{-lambda_j t}
  a_p(t) = a_p(0) e^{-mu t} + v_p(s) / (Ss V) sum_j c_j (e^{-lambda_j t} - e^{-mu t}) / (mu - lambda_j)
(the limit t e^{-mu t} when mu = lambda_j).  A constant rate Q is c = Q, lambda = 0:
  v_p(s) Q / (Ss V) (1 - e^{-mu t}) / mu, and t v_p(s) Q / (Ss V) for a zero mode (all faces Neumann).

This is a closed form (textbook separation of variables) and pins O1.
"""
from __future__ import annotations

import numpy as np


def _axis_basis(n, code):
    j = np.arange(n) + 0.5
    if code == 0:
        p = np.arange(1, n + 1)
        V = np.sin(np.outer(j, p) * np.pi / n)
    else:
        p = np.arange(0, n)
        V = np.cos(np.outer(j, p) * np.pi / n)
    V /= np.linalg.norm(V, axis=0)        # sqrt(2/n), except sqrt(1/n) for p = n (D) and p = 0 (N)
    lam = 4.0 * np.sin(p * np.pi / (2.0 * n)) ** 2
    return V, lam


def _duhamel(mu, lam, t):
    """int_0^t e^{-mu (t - s)} e^{-lam s} ds, elementwise over the mode array mu."""
    d = mu - lam
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        near = np.abs(d) * t < 1e-8
        safe = np.where(near, 1.0, d)
        # (e^{-lam t} - e^{-mu t}) / (mu - lam) = e^{-lam t} (1 - e^{-d t}) / d
        g = np.exp(-lam * t) * (-np.expm1(-d * t)) / safe
        g_near = t * np.exp(-lam * t) * (1.0 - 0.5 * d * t)
    return np.where(near, g_near, g)


def heads(prob, times=None):
    """h[ns][nr][nt] for a homogeneous problem (uniform kappa, Ss)."""
    from . import source
    kap = float(np.asarray(prob.kappa).ravel()[0])
    ss = float(np.asarray(prob.Ss).ravel()[0])
    assert np.allclose(prob.kappa, kap) and np.allclose(prob.Ss, ss)
    bc = prob.bc
    for a in range(3):
        assert bc[2 * a] == bc[2 * a + 1], "closed form needs the same BC at both ends of an axis"
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    Vx, lx = _axis_basis(nx, bc[0])
    Vy, ly = _axis_basis(ny, bc[2])
    Vz, lz = _axis_basis(nz, bc[4])
    vol = dx * dy * dz
    kx, ky, kz = kap * dy * dz / dx, kap * dx * dz / dy, kap * dx * dy / dz
    lam = (kx * lx[None, None, :] + ky * ly[None, :, None] + kz * lz[:, None, None])  # [pz, py, px]
    mu = lam / (ss * vol)
    times = prob.times if times is None else np.asarray(times)
    # initial-state coefficients a_p(0) = v_p . phi_0 (separable basis: one tensor contraction)
    p0 = source.initial_state(prob).reshape(nz, ny, nx)
    a0 = np.einsum("kji,kc,jb,ia->cba", p0, Vz, Vy, Vx)

    def unravel(c):
        i = c % nx; jj = (c // nx) % ny; k = c // (nx * ny)
        return i, jj, k

    h = np.zeros((len(prob.src_cells), len(prob.rec_cells), len(times)))
    for si, sc in enumerate(prob.src_cells):
        i, j, k = unravel(int(sc))
        cs = Vz[k][:, None, None] * Vy[j][None, :, None] * Vx[i][None, None, :]
        amp, rates = source.terms(prob, si)
        for ri, rc in enumerate(prob.rec_cells):
            a, b, c = unravel(int(rc))
            cr = Vz[c][:, None, None] * Vy[b][None, :, None] * Vx[a][None, None, :]
            coef = cs * cr / (ss * vol)
            for ti, t in enumerate(times):
                g = sum(cj * _duhamel(mu, lj, t) for cj, lj in zip(amp, rates))
                h[si, ri, ti] = np.sum(coef * g) + np.sum(cr * a0 * np.exp(-mu * t))
    return h
