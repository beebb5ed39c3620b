"""O1: Laplace-transform solution with a direct complex LU per shift.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

For each output time t and each upper-half contour node z_k (Sec. 2.2):
    x_k = (K + z_k M)^{-1} (q_hat_s(z_k) e_s + M phi_0)
(the Laplace transform of the semi-discrete system, Sec. 2.1, with the two
right-hand sides [b, M phi_0] of Sec. 3; q_hat = Q / z for a constant rate
switched on at t = 0, sum_j a_j / (z + lambda_j) for an exponential-sum rate,
see oracle/source.py), and
    phi(t) = 2 Re sum_k w_k x_k        (Eq. half),
    h[s, r, t] = phi_s(t)[receiver r].
This is the 'Direct' solver of the paper's timing comparison (Sec. 5.3).

Pinned by the eigen-expansion closed form (O2, exact for homogeneous boxes),
by Crank-Nicolson (O3) and by the matrix exponential of the ODE on small
grids in tests/test_oracle_forward.py and tests/test_oracle_initial_rates.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import contour, fv, source


def shifted_solve(K, m, z, B):
    """Solve (K + z M) X = B with SuperLU (complex)."""
    A = (K + z * sp.diags(m)).astype(np.complex128).tocsc()
    lu = spla.splu(A)
    return lu.solve(np.asarray(B, dtype=np.complex128))


def forward(prob, return_fields: bool = False, sources=None, times=None):
    """Measurements h[ns][nr][nt] (and optionally fields phi[ns][nt][N])."""
    K, m = fv.assemble(prob)
    src = list(range(len(prob.src_cells))) if sources is None else list(sources)
    times = prob.times if times is None else np.asarray(times)
    N = prob.ncell
    mphi0 = m * source.initial_state(prob)
    h = np.zeros((len(src), len(prob.rec_cells), len(times)))
    fields = np.zeros((len(src), len(times), N)) if return_fields else None
    for it, t in enumerate(times):
        z, w = contour.nodes_weights(t, prob.Nz, half=True)
        acc = np.zeros((N, len(src)), dtype=np.complex128)
        for zk, wk in zip(z, w):
            B = np.zeros((N, len(src)), dtype=np.complex128)
            for j, s in enumerate(src):
                B[prob.src_cells[s], j] = source.q_hat(prob, s, zk)
                B[:, j] += mphi0
            X = shifted_solve(K, m, zk, B)
            acc += wk * X
        phi = 2.0 * acc.real
        h[:, :, it] = phi[prob.rec_cells, :].T
        if return_fields:
            fields[:, it, :] = phi.T
    return (h, fields) if return_fields else h


def shifted_solutions(prob, t, s):
    """All x_k = (K + z_k M)^{-1} b_s for one time (unscaled by q_hat)."""
    K, m = fv.assemble(prob)
    z, w = contour.nodes_weights(t, prob.Nz, half=True)
    b = fv.rhs(prob, s)
    return z, w, np.stack([shifted_solve(K, m, zk, b) for zk in z])
