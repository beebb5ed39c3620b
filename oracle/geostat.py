"""Quasi-linear geostatistical inversion (Sec. 5.1, Algorithm 2), FP64 on the CPU.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

Unknown: s = log kappa per cell (the paper inverts log transmissivity), prior
s ~ N(X beta, Q) with X = the column of ones (one unknown drift, p = 1) and Q the
exponential covariance Q_ij = sigma2 exp(-|x_i - x_j| / ell) between cell
centres (Sec. 5.1 names the exponential kernel of the Matern family); data
y = h(s) + eps, eps ~ N(0, R), R diagonal.  One iteration of Algorithm 2 at s_k:

    J_k = d h / d s at s_k                                   (O4, the log-kappa half)
    [ J_k Q J_k^T + R   J_k X ] [ xi   ]   [ y - h(s_k) + J_k s_k ]
    [ (J_k X)^T          0    ] [ beta ] = [ 0                    ]
    s_{k+1} = X beta + Q J_k^T xi.

The dense Q and the dense saddle-point solve are the plain definitions (the GPU
path forms Q J^T by FFT on the circulant embedding of the covariance).

Pinned by tests/test_oracle_geostat.py: for a linear forward map one iteration
gives the minimiser of the MAP objective with beta profiled out (computed here
independently from the normal equations of the objective); at a fixed point of
the iteration on the nonlinear problem the objective's first-order conditions
hold (xi = R^{-1}(y - h(s)), X^T Q^{-1}(s - X beta) = 0).
"""
from __future__ import annotations

import copy

import numpy as np

from . import adjoint, direct


def cell_centres(prob):
    """[N, 3] cell-centre coordinates (x fastest, the grid's cell order)."""
    k, j, i = np.meshgrid(np.arange(prob.nz), np.arange(prob.ny), np.arange(prob.nx), indexing="ij")
    return np.stack([(i.ravel() + 0.5) * prob.dx, (j.ravel() + 0.5) * prob.dy, (k.ravel() + 0.5) * prob.dz], 1)


def exp_covariance(prob, sigma2: float, ell: float):
    """Dense Q_ij = sigma2 exp(-|x_i - x_j| / ell)."""
    x = cell_centres(prob)
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    return sigma2 * np.exp(-d / ell)


def with_log_kappa(prob, s):
    p = copy.copy(prob)
    p.kappa = np.exp(np.asarray(s, dtype=np.float64)).reshape(prob.kappa.shape)
    return p


def forward_and_jacobian(prob, s):
    """h(s) flattened in [s][r][t] order and J = d h / d log kappa [Ny, N]."""
    p = with_log_kappa(prob, s)
    h = direct.forward(p).ravel()
    J = adjoint.jacobian(p)[:, :, :, 0, :].reshape(h.size, prob.ncell)
    return h, J


def gn_step(Q, R, X, y, s, h, J):
    """One iteration of Algorithm 2 from s with h = h(s), J = J(s); returns (s_next, beta, xi)."""
    ny = y.size
    p = X.shape[1]
    JX = J @ X
    A = np.zeros((ny + p, ny + p))
    A[:ny, :ny] = J @ Q @ J.T + np.diag(R)
    A[:ny, ny:] = JX
    A[ny:, :ny] = JX.T
    rhs = np.concatenate([y - h + J @ s, np.zeros(p)])
    sol = np.linalg.solve(A, rhs)
    xi, beta = sol[:ny], sol[ny:]
    return X @ beta + Q @ (J.T @ xi), beta, xi


def gauss_newton(prob, y, R, sigma2, ell, s0, iters: int = 10, tol: float = 1e-10):
    """Algorithm 2 from s0; stops when the step is below tol (relative); returns (s, history)."""
    Q = exp_covariance(prob, sigma2, ell)
    X = np.ones((prob.ncell, 1))
    s = np.asarray(s0, dtype=np.float64).copy()
    hist = []
    for _ in range(iters):
        h, J = forward_and_jacobian(prob, s)
        s_new, beta, xi = gn_step(Q, R, X, y, s, h, J)
        step = np.linalg.norm(s_new - s) / max(np.linalg.norm(s_new), 1e-300)
        hist.append(dict(step=step, beta=beta.copy(), misfit=float(np.sum((y - h) ** 2 / R))))
        s = s_new
        if step < tol:
            break
    return s, hist
