"""Algorithm 1 (flexible FOM/GMRES for shifted systems), with exact
shift-and-invert preconditioners factorised by sparse LU (Sec. 3).

Given K, M, b, preconditioner shifts tau_j and shifts z_k:
  v_1 = b / beta,  beta = ||b||
  for j = 1, 2, ...:
      solve (K + tau_j M) u_j = v_j
      s_j = M u_j
      Arnoldi (modified Gram-Schmidt): h_ij = v_i^H s_j, s_j -= h_ij v_i
      h_{j+1,j} = ||s_j||, v_{j+1} = s_j / h_{j+1,j}
      for every unconverged shift z_k:
          Hbar(z_k; T_j) = [I; 0] + Hbar_j (z_k I - T_j)      (Eq. shiftedarnoldimod)
          GMRES: y = argmin || beta e_1 - Hbar(z_k; T_j) y ||
          (FOM : H(z_k; T_j) y = beta e_1)
          converged when the projected residual <= tol * beta
  x(z_k) = U_j y(z_k).
(The printed listing's inner loop writes h_ij := s_j^* v_i and
s_j := s_j - h_ij v_j; the Arnoldi process it describes takes v_i^H s_j and
subtracts h_ij v_i, which is what is done here.)

Stopping rules.  "shift": each shift stops on its own projected residual
(GMRES: the least-squares residual; FOM: |eta_k|, below).  "quadrature":
the shifts of one output time stop together once the quadrature-weighted sum
sum_k |omega_k| rho_k <= tol beta sum_k |omega_k| (omega_k = w_k q_hat(z_k),
rho_k the shift's projected residual), the a-posteriori bound on the
residual of the quadrature sum in Sec. 3.1 (Proposition 1 and the remark
after its proof: ||r_m|| <= sum_k |w_k| |eta_k|).  For FOM the projected
residual is |eta_k| = |h_{j+1,j} (z_k - tau_j) e_j^T H_j(z_k; T_j)^{-1} beta e_1|,
and b - (K + z_k M) x_k = -eta_k v_{j+1} exactly (the proof of Proposition 1).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

Pinned by tests/test_oracle_krylov.py: solutions equal the direct LU (O1)
to the tolerance, the Arnoldi identity (K + zM) U = V Hbar(z; T) holds
to rounding, and |eta_k| equals the FOM true residual.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve(K, m, b, zs, taus, tol=1e-10, maxit=300, variant="gmres", true_residual=False, stop="shift",
          weights=None, time_of=None, return_residuals=False):
    """Return (X [nshift, N], iterations used, per-shift iteration of convergence) and, with
    return_residuals, the last projected residual of every shift (|eta_k| for FOM) relative to beta.
    stop="quadrature" needs weights (|omega_k| per shift) and time_of (output-time label per shift)."""
    zs = np.asarray(zs, dtype=np.complex128)
    M = sp.diags(m)
    N = K.shape[0]
    beta = np.linalg.norm(b)
    V = [b.astype(np.complex128) / beta]
    U = []
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    T = []
    lus = {}
    conv = np.full(len(zs), -1)
    Y = [None] * len(zs)
    pres = np.ones(len(zs))
    if stop == "quadrature":
        weights = np.asarray(weights, dtype=np.float64)
        time_of = np.asarray(time_of)
    j = 0
    for j in range(maxit):
        tau = complex(taus[j])
        if tau not in lus:
            lus[tau] = spla.splu((K + tau * M).astype(np.complex128).tocsc())
        u = lus[tau].solve(V[j])
        U.append(u)
        T.append(tau)
        s = m * u
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], s)
            s = s - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(s)
        breakdown = H[j + 1, j] == 0
        V.append(s / (H[j + 1, j] if not breakdown else 1.0))
        Hb = H[: j + 2, : j + 1]
        Tj = np.array(T)
        e1 = np.zeros(j + 2, dtype=np.complex128)
        e1[0] = beta
        for k, z in enumerate(zs):
            if conv[k] >= 0:
                continue
            Hz = np.eye(j + 2, j + 1, dtype=np.complex128) + Hb * (z - Tj)[None, :]
            if variant == "fom":
                y = np.linalg.solve(Hz[: j + 1, :], e1[: j + 1])
            else:
                y = np.linalg.lstsq(Hz, e1, rcond=None)[0]
            res = np.linalg.norm(e1 - Hz @ y)
            Y[k] = y
            pres[k] = res / beta
            if stop == "shift" and (res <= tol * beta or breakdown):
                conv[k] = j + 1
        if stop == "quadrature":
            for t in np.unique(time_of):
                sel = (time_of == t) & (conv < 0)
                if not np.any(sel):
                    continue
                if np.sum(weights[sel] * pres[sel]) <= tol * np.sum(weights[sel]) or breakdown:
                    conv[sel] = j + 1
        if np.all(conv >= 0):
            break
    Um = np.array(U).T
    X = np.stack([Um[:, : len(Y[k])] @ Y[k] for k in range(len(zs))])
    if return_residuals:
        return X, j + 1, conv, pres
    return X, j + 1, conv


def arnoldi_identity_error(K, m, b, z, taus, nit):
    """max over columns of ||(K + zM) U - V Hbar(z; T)|| / ||V Hbar||."""
    M = sp.diags(m)
    beta = np.linalg.norm(b)
    V = [b.astype(np.complex128) / beta]
    U, T = [], []
    H = np.zeros((nit + 1, nit), dtype=np.complex128)
    for j in range(nit):
        u = spla.spsolve((K + taus[j] * M).astype(np.complex128).tocsc(), V[j])
        U.append(u); T.append(taus[j])
        s = m * u
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], s)
            s = s - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(s)
        V.append(s / H[j + 1, j])
    Um = np.array(U).T
    Vm = np.array(V).T
    Hz = np.eye(nit + 1, nit) + H * (z - np.array(T))[None, :]
    lhs = (K + z * M) @ Um
    rhs = Vm @ Hz
    return np.max(np.linalg.norm(lhs - rhs, axis=0) / np.linalg.norm(rhs, axis=0))
