"""Cell-centred finite-volume restatement of the semi-discrete system
M phi' + K phi = q(t) b (Sec. 2.1, the weak form and Eq. for K_ij, M_ij).

The paper discretises with P1 finite elements; this oracle (like the CUDA
path) uses the cell-centred two-point-flux finite-volume scheme:

* interior face between cells a, b (same size):
  T_f = (area / dist) * 2 kappa_a kappa_b / (kappa_a + kappa_b)  (harmonic mean)
* Dirichlet boundary face (ghost half a cell away, phi = 0 there):
  T_f = 2 kappa_c area / dist
* Neumann face: T_f = 0
* linearised water-table face (Sec. 2.1, the boundary term (S_y d phi/dt, psi) of the weak
  form): no flux, T_f = 0, and S_y,c times the face area joins the cell's storage
* K = sum_f T_f (e_a - e_b)(e_a - e_b)^T + sum_{Dirichlet f} T_f e_c e_c^T
* M = diag(Ss_c * V_c + sum_{water-table f of c} Sy_c A_f),  b = Q e_source.

Pinned by: the eigen-expansion closed form (tests/test_oracle_forward.py),
symmetry/positivity of K, and the row-sum identity (K 1 = boundary terms).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def face_transmissibilities(kappa, dx, dy, dz, bc):
    """Return dict with interior face arrays and boundary-face arrays.

    tx[k, j, i] for the face between cell (i, j, k) and (i+1, j, k),
    shape (nz, ny, nx-1); likewise ty (nz, ny-1, nx), tz (nz-1, ny, nx).
    Boundary arrays bx0, bx1 (nz, ny), by0, by1 (nz, nx), bz0, bz1 (ny, nx):
    the Dirichlet face transmissibility (0 for Neumann faces).
    """
    k = np.asarray(kappa, dtype=np.float64)
    ax, ay, az = dy * dz, dx * dz, dx * dy

    def harm(a, b):
        return 2.0 * a * b / (a + b)

    tx = ax / dx * harm(k[:, :, :-1], k[:, :, 1:])
    ty = ay / dy * harm(k[:, :-1, :], k[:, 1:, :])
    tz = az / dz * harm(k[:-1, :, :], k[1:, :, :])
    d = lambda code: 1.0 if code == 0 else 0.0
    bx0 = d(bc[0]) * 2.0 * k[:, :, 0] * ax / dx
    bx1 = d(bc[1]) * 2.0 * k[:, :, -1] * ax / dx
    by0 = d(bc[2]) * 2.0 * k[:, 0, :] * ay / dy
    by1 = d(bc[3]) * 2.0 * k[:, -1, :] * ay / dy
    bz0 = d(bc[4]) * 2.0 * k[0, :, :] * az / dz
    bz1 = d(bc[5]) * 2.0 * k[-1, :, :] * az / dz
    return dict(tx=tx, ty=ty, tz=tz, bx0=bx0, bx1=bx1, by0=by0, by1=by1, bz0=bz0, bz1=bz1)


def assemble(prob):
    """Assemble (K as CSR float64, m = diag(M) as float64 vector)."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    N = nx * ny * nz
    f = face_transmissibilities(prob.kappa, prob.dx, prob.dy, prob.dz, prob.bc)
    idx = np.arange(N).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros((nz, ny, nx))

    def add_pairs(a, b, t):
        a = a.ravel(); b = b.ravel(); t = t.ravel()
        rows.extend([a, b]); cols.extend([b, a]); vals.extend([-t, -t])

    add_pairs(idx[:, :, :-1], idx[:, :, 1:], f["tx"])
    diag[:, :, :-1] += f["tx"]; diag[:, :, 1:] += f["tx"]
    add_pairs(idx[:, :-1, :], idx[:, 1:, :], f["ty"])
    diag[:, :-1, :] += f["ty"]; diag[:, 1:, :] += f["ty"]
    if nz > 1:
        add_pairs(idx[:-1, :, :], idx[1:, :, :], f["tz"])
        diag[:-1, :, :] += f["tz"]; diag[1:, :, :] += f["tz"]
    diag[:, :, 0] += f["bx0"]; diag[:, :, -1] += f["bx1"]
    diag[:, 0, :] += f["by0"]; diag[:, -1, :] += f["by1"]
    diag[0, :, :] += f["bz0"]; diag[-1, :, :] += f["bz1"]
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(diag.ravel())
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    m = (np.asarray(prob.Ss, dtype=np.float64) * (prob.dx * prob.dy * prob.dz)).ravel()
    m = m + water_table_storage(prob)
    return K, m


def water_table_storage(prob):
    """Per cell: sum over its water-table faces of S_y,c times the face area (zeros if none)."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    add = np.zeros((nz, ny, nx))
    if not any(code == 2 for code in prob.bc):
        return add.ravel()
    sy = np.asarray(prob.Sy, dtype=np.float64).reshape(nz, ny, nx)
    ax, ay, az = prob.dy * prob.dz, prob.dx * prob.dz, prob.dx * prob.dy
    sel = [(0, (slice(None), slice(None), 0), ax), (1, (slice(None), slice(None), -1), ax),
           (2, (slice(None), 0, slice(None)), ay), (3, (slice(None), -1, slice(None)), ay),
           (4, (0, slice(None), slice(None)), az), (5, (-1, slice(None), slice(None)), az)]
    for face, idx, area in sel:
        if prob.bc[face] == 2:
            add[idx] += sy[idx] * area
    return add.ravel()


def rhs(prob, s):
    """b = Q_s e_{cell(s)} (point source, Sec. 2.1 b_j = (delta(x - x_s), u_j))."""
    b = np.zeros(prob.ncell)
    b[prob.src_cells[s]] = prob.Q[s]
    return b
