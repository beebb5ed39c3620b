"""Block flexible GMRES for shifted systems: Algorithm 1 (Sec. 3) with the right-hand sides of
several sources taken as one block, the block Krylov variant Sec. 6 leaves to future work.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

For B = [b_1 .. b_p] (N x p) with B = V_1 beta (thin QR), preconditioner shifts tau_j and shifts z_k:
  for j = 1, 2, ...:
      U_j = (K + tau_j M)^{-1} V_j                 (p solves, exact LU here)
      S = M U_j
      block Gram-Schmidt, twice: H_ij = V_i^H S, S -= V_i H_ij   (i <= j)
      S = V_{j+1} H_{j+1,j}                        (thin QR; H_{j+1,j} upper triangular)
  so that (K + z M) U_m = V_{m+1} Hbar(z),  Hbar(z) = [I; 0] + Hbar_m (z I - T_m (x) I_p),
and for every shift  Y(z) = argmin || E_1 beta - Hbar(z) Y ||_F  (p right-hand sides at once),
X(z) = U_m Y(z).  Right-hand side q of shift k converges when its column's residual is
<= tol ||b_q||.  With p = 1 this is Algorithm 1 exactly.

Pinned by tests/test_oracle_block.py: p = 1 reproduces the oracle's Algorithm 1, the block
Arnoldi identity holds to rounding, and the solutions equal the direct LU to the tolerance.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve(K, m, B, zs, taus, tol=1e-10, maxit=200):
    """Return (X [nshift][N][p], iterations, conv [nshift][p] iteration of convergence, -1 if not),
    and the final per-(shift, rhs) relative residuals."""
    B = np.asarray(B, dtype=np.complex128)
    N, p = B.shape
    zs = np.asarray(zs, dtype=np.complex128)
    M = sp.diags(m)
    V1, beta = np.linalg.qr(B)
    bn = np.linalg.norm(B, axis=0)
    V = [V1]
    U = []
    T = []
    H = np.zeros(((maxit + 1) * p, maxit * p), dtype=np.complex128)
    lus = {}
    conv = np.full((len(zs), p), -1)
    res = np.ones((len(zs), p))
    j = 0
    for j in range(maxit):
        tau = complex(taus[j])
        if tau not in lus:
            lus[tau] = spla.splu((K + tau * M).astype(np.complex128).tocsc())
        Uj = lus[tau].solve(V[j])
        U.append(Uj)
        T.append(tau)
        S = m[:, None] * Uj
        for _ in range(2):
            for i in range(j + 1):
                Hij = V[i].conj().T @ S
                H[i * p:(i + 1) * p, j * p:(j + 1) * p] += Hij
                S = S - V[i] @ Hij
        Vn, Rn = np.linalg.qr(S)
        H[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Rn
        V.append(Vn)
        n = (j + 1) * p
        Hb = H[:n + p, :n]
        dz_base = np.repeat(np.array(T), p)
        E1 = np.zeros((n + p, p), dtype=np.complex128)
        E1[:p, :] = beta
        for k, z in enumerate(zs):
            Hz = np.eye(n + p, n, dtype=np.complex128) + Hb * (z - dz_base)[None, :]
            Y = np.linalg.lstsq(Hz, E1, rcond=None)[0]
            R = E1 - Hz @ Y
            for q in range(p):
                if conv[k, q] >= 0:
                    continue
                res[k, q] = np.linalg.norm(R[:, q]) / bn[q]
                if res[k, q] <= tol:
                    conv[k, q] = j + 1
        if np.all(conv >= 0):
            break
    Um = np.concatenate(U, axis=1)
    X = np.zeros((len(zs), N, p), dtype=np.complex128)
    for k in range(len(zs)):
        # each right-hand side takes its coefficients at the iteration where it converged
        for q in range(p):
            it = conv[k, q] if conv[k, q] > 0 else j + 1
            n = it * p
            Hz = np.eye(n + p, n, dtype=np.complex128) + H[:n + p, :n] * (zs[k] - np.repeat(np.array(T[:it]), p))[None, :]
            E1 = np.zeros((n + p, p), dtype=np.complex128)
            E1[:p, :] = beta
            y = np.linalg.lstsq(Hz, E1[:, q], rcond=None)[0]
            X[k, :, q] = Um[:, :n] @ y
    return X, j + 1, conv, res


def arnoldi_identity_error(K, m, B, z, taus, nit):
    """max over columns of ||(K + z M) U - V Hbar(z)|| / ||V Hbar(z)|| after nit block iterations."""
    B = np.asarray(B, dtype=np.complex128)
    N, p = B.shape
    M = sp.diags(m)
    V1, _ = np.linalg.qr(B)
    V, U, T = [V1], [], []
    H = np.zeros(((nit + 1) * p, nit * p), dtype=np.complex128)
    for j in range(nit):
        Uj = spla.spsolve((K + taus[j] * M).astype(np.complex128).tocsc(), V[j])
        Uj = Uj.reshape(N, p)
        U.append(Uj); T.append(taus[j])
        S = m[:, None] * Uj
        for _ in range(2):
            for i in range(j + 1):
                Hij = V[i].conj().T @ S
                H[i * p:(i + 1) * p, j * p:(j + 1) * p] += Hij
                S = S - V[i] @ Hij
        Vn, Rn = np.linalg.qr(S)
        H[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Rn
        V.append(Vn)
    Um = np.concatenate(U, axis=1)
    Vm = np.concatenate(V, axis=1)
    Hz = np.eye((nit + 1) * p, nit * p) + H * (z - np.repeat(np.array(T), p))[None, :]
    lhs = (K + z * M) @ Um
    rhs = Vm @ Hz
    return float(np.max(np.linalg.norm(lhs - rhs, axis=0) / np.linalg.norm(rhs, axis=0)))
