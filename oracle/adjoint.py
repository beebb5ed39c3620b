"""O4: Laplace-domain adjoint Jacobian of the measurements (Sec. 5.2).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

Measurement h_{s,r}(t) = e_r^T phi_s(t), phi_s(t) = 2 Re sum_k w_k qhat_s(z_k)
xhat_{s,k}, xhat_{s,k} = A_k^{-1} e_{cell(s)}, A_k = K + z_k M, with
qhat_s(z) = Q_s / z for a constant rate (oracle/source.py for exponential
sums) and phi_0 = 0.  Since w_k,
z_k do not depend on the parameters, and A_k is complex symmetric (so the
adjoint field uses a transpose, not a conjugate transpose):

  dh_{s,r}(t)/dp = -2 Re sum_k w_k qhat_s(z_k) psi_{r,k}^T (dK/dp + z_k dM/dp) xhat_{s,k},
  psi_{r,k} = A_k^{-1} e_{cell(r)}

(the discrete counterpart of the sensitivity formula of Sec. 5.2 with the
adjoint problem driven by the point measurement).  With p = log kappa_c:
  psi^T dK x = sum over interior faces f of c:
                 T_f kappa_o / (kappa_c + kappa_o) (psi_c - psi_o)(x_c - x_o)
             + sum over Dirichlet faces of c: T_f psi_c x_c
and with p = log Ss_c:  psi^T z dM x = z Ss_c V_c psi_c x_c (the storage of a water-table face,
S_y A_f, does not depend on Ss).

Pinned by tests/test_oracle_adjoint.py: central finite differences of O1 on
tiny grids, the scale invariant sum_c (dh/dlog kappa_c + dh/dlog Ss_c) = -h,
and the time-scaling invariant sum_c dh/dlog kappa_c = -h + t dh/dt.
"""
from __future__ import annotations

import copy

import numpy as np

from . import contour, direct, fv, source


def face_weights(prob):
    """Per-face derivative weights dT_f/dlog kappa for both adjacent cells."""
    f = fv.face_transmissibilities(prob.kappa, prob.dx, prob.dy, prob.dz, prob.bc)
    k = prob.kappa
    out = {}
    for name, sl_a, sl_b in (("tx", (slice(None), slice(None), slice(None, -1)), (slice(None), slice(None), slice(1, None))),
                             ("ty", (slice(None), slice(None, -1), slice(None)), (slice(None), slice(1, None), slice(None))),
                             ("tz", (slice(None, -1), slice(None), slice(None)), (slice(1, None), slice(None), slice(None)))):
        ka, kb = k[sl_a], k[sl_b]
        T = f[name]
        out[name] = (T * kb / (ka + kb), T * ka / (ka + kb), sl_a, sl_b)
    out["bnd"] = f
    return out


def _bilinear_terms(prob, fw, psi, x):
    """Per-cell psi^T (dK/dlog kappa_c) x, shape (nz, ny, nx), complex."""
    nz, ny, nx = prob.nz, prob.ny, prob.nx
    P = psi.reshape(nz, ny, nx)
    X = x.reshape(nz, ny, nx)
    g = np.zeros((nz, ny, nx), dtype=np.complex128)
    for name in ("tx", "ty", "tz"):
        wa, wb, sa, sb = fw[name]
        if wa.size == 0:
            continue
        prod = (P[sa] - P[sb]) * (X[sa] - X[sb])
        g[sa] += wa * prod
        g[sb] += wb * prod
    b = fw["bnd"]
    g[:, :, 0] += b["bx0"] * P[:, :, 0] * X[:, :, 0]
    g[:, :, -1] += b["bx1"] * P[:, :, -1] * X[:, :, -1]
    g[:, 0, :] += b["by0"] * P[:, 0, :] * X[:, 0, :]
    g[:, -1, :] += b["by1"] * P[:, -1, :] * X[:, -1, :]
    g[0, :, :] += b["bz0"] * P[0, :, :] * X[0, :, :]
    g[-1, :, :] += b["bz1"] * P[-1, :, :] * X[-1, :, :]
    return g.ravel()


def jacobian(prob):
    """J[ns][nr][nt][2][N]: d h / d log kappa (index 0), d h / d log Ss (1)."""
    assert not np.any(source.initial_state(prob)), "the adjoint here assumes phi_0 = 0"
    K, m = fv.assemble(prob)
    mss = (np.asarray(prob.Ss, dtype=np.float64) * (prob.dx * prob.dy * prob.dz)).ravel()   # dM / dlog Ss
    N = prob.ncell
    ns, nr, nt = len(prob.src_cells), len(prob.rec_cells), len(prob.times)
    fw = face_weights(prob)
    J = np.zeros((ns, nr, nt, 2, N))
    E_s = np.zeros((N, ns)); E_s[prob.src_cells, np.arange(ns)] = 1.0
    E_r = np.zeros((N, nr)); E_r[prob.rec_cells, np.arange(nr)] = 1.0
    for it, t in enumerate(prob.times):
        z, w = contour.nodes_weights(t, prob.Nz, half=True)
        for zk, wk in zip(z, w):
            Xs = direct.shifted_solve(K, m, zk, E_s)      # [N, ns]
            Ps = direct.shifted_solve(K, m, zk, E_r)      # [N, nr]
            for s in range(ns):
                coef = wk * source.q_hat(prob, s, zk)
                for r in range(nr):
                    gk = _bilinear_terms(prob, fw, Ps[:, r], Xs[:, s])
                    gs = zk * mss * Ps[:, r] * Xs[:, s]
                    J[s, r, it, 0] += -2.0 * np.real(coef * gk)
                    J[s, r, it, 1] += -2.0 * np.real(coef * gs)
    return J


def dh_dt(prob):
    """Time derivative of the measurements: 2 Re sum_k w_k z_k x_k (Q/z_k)."""
    K, m = fv.assemble(prob)
    ns, nr, nt = len(prob.src_cells), len(prob.rec_cells), len(prob.times)
    N = prob.ncell
    E_s = np.zeros((N, ns)); E_s[prob.src_cells, np.arange(ns)] = prob.Q
    out = np.zeros((ns, nr, nt))
    for it, t in enumerate(prob.times):
        z, w = contour.nodes_weights(t, prob.Nz, half=True)
        acc = np.zeros((N, ns), dtype=np.complex128)
        for zk, wk in zip(z, w):
            acc += wk * direct.shifted_solve(K, m, zk, E_s)   # z_k * (Q/z_k) = Q
        out[:, :, it] = 2.0 * acc.real[prob.rec_cells, :].T
    return out


def fd_jacobian(prob, cells, which: int, delta: float = 1e-4):
    """Central differences of O1 w.r.t. log kappa (which=0) or log Ss (1)
    at the given cells: returns [ns][nr][nt][len(cells)]."""
    out = np.zeros((len(prob.src_cells), len(prob.rec_cells), len(prob.times), len(cells)))
    for ci, c in enumerate(cells):
        hs = []
        for sgn in (+1.0, -1.0):
            p = copy.copy(prob)
            kap = prob.kappa.copy().ravel(); ss = prob.Ss.copy().ravel()
            if which == 0:
                kap[c] *= np.exp(sgn * delta)
            else:
                ss[c] *= np.exp(sgn * delta)
            p.kappa = kap.reshape(prob.kappa.shape); p.Ss = ss.reshape(prob.Ss.shape)
            hs.append(direct.forward(p))
        out[..., ci] = (hs[0] - hs[1]) / (2.0 * delta)
    return out
