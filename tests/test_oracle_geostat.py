"""Pins for the oracle's quasi-linear geostatistical inversion (Sec. 5.1, Algorithm 2).

* Linear forward map h(s) = H s: one iteration must give the minimiser of the MAP objective
  1/2 ||y - H s||^2_{R^-1} + 1/2 ||s - X beta||^2_{Q^-1} over (s, beta), computed here from the
  objective's normal equations (with Q^-1, not the cokriging system the algorithm solves).
* Nonlinear (the aquifer): at the fixed point of the iteration the first-order conditions of the
  objective hold: xi = R^-1 (y - h(s)) (from -J^T R^-1 (y - h) + Q^-1 (s - X beta) = 0 and
  s - X beta = Q J^T xi), and the data misfit falls from the prior mean to the estimate."""
import numpy as np

import workloads as W
from oracle import geostat


def test_one_iteration_is_the_map_estimate_for_a_linear_map():
    rng = np.random.default_rng(0)
    p = W.random_problem(6, 5, 1, variance=0.0, seed=1, ns=1, nr=1, nt=1)
    N, ny = p.ncell, 12
    Q = geostat.exp_covariance(p, 0.8, 30.0)
    X = np.ones((N, 1))
    H = rng.standard_normal((ny, N))
    R = rng.uniform(0.01, 0.05, ny)
    y = rng.standard_normal(ny)
    s0 = rng.standard_normal(N)
    s1, beta, xi = geostat.gn_step(Q, R, X, y, s0, H @ s0, H)
    # normal equations of the objective in (s, beta)
    Qi = np.linalg.inv(Q)
    A = np.zeros((N + 1, N + 1))
    A[:N, :N] = H.T @ np.diag(1.0 / R) @ H + Qi
    A[:N, N:] = -Qi @ X
    A[N:, :N] = -(Qi @ X).T
    A[N:, N:] = X.T @ Qi @ X
    rhs = np.concatenate([H.T @ (y / R), [0.0]])
    sol = np.linalg.solve(A, rhs)
    assert np.linalg.norm(s1 - sol[:N]) / np.linalg.norm(sol[:N]) < 1e-9
    assert abs(beta[0] - sol[N]) <= 1e-9 * max(abs(sol[N]), 1.0)


def test_fixed_point_satisfies_the_first_order_conditions():
    p = W.random_problem(8, 8, 1, variance=0.0, seed=2, ns=2, nr=4, nt=2, Nz=16)
    sigma2, ell = 0.5, 40.0
    rng = np.random.default_rng(3)
    Q = geostat.exp_covariance(p, sigma2, ell)
    Lq = np.linalg.cholesky(Q + 1e-12 * np.eye(p.ncell))
    s_true = np.log(1e-4) + Lq @ rng.standard_normal(p.ncell)
    h_true, _ = geostat.forward_and_jacobian(p, s_true)
    scale = np.abs(h_true).max()
    R = np.full(h_true.size, (1e-3 * scale) ** 2)
    y = h_true + np.sqrt(R) * rng.standard_normal(h_true.size)
    s0 = np.full(p.ncell, np.log(1e-4))
    s, hist = geostat.gauss_newton(p, y, R, sigma2, ell, s0, iters=30, tol=1e-10)
    assert hist[-1]["step"] < 1e-10        # linear convergence (ratio about 0.3 here)
    h, J = geostat.forward_and_jacobian(p, s)
    X = np.ones((p.ncell, 1))
    _, beta, xi = geostat.gn_step(Q, R, X, y, s, h, J)
    target = (y - h) / R
    assert np.linalg.norm(xi - target) <= 1e-6 * np.linalg.norm(target)
    assert hist[-1]["misfit"] < 0.1 * hist[0]["misfit"]
