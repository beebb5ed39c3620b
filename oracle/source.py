"""Source time functions and their Laplace transforms (Sec. 2.1-2.2).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

The method needs sources that separate in space and time, f = q(t) b, with a
Laplace transform q_hat(z) that is known for every contour node.  Sec. 2.2
points to exponential sums, q(t) ~ sum_j a_j exp(-lambda_j t) (fitted by
Prony's method when q is given otherwise), whose transform is
    q_hat(z) = sum_j a_j / (z + lambda_j).
A constant rate Q switched on at t = 0 is the one-term sum with lambda = 0:
q_hat(z) = Q / z.  The poles -lambda_j <= 0 lie left of the Talbot contour,
which crosses the real axis at a positive abscissa, so the quadrature of
Sec. 2.2 applies unchanged.

Initial state (Sec. 3, the two right-hand sides [b, M phi_0]): the Laplace
transform of M phi' + K phi = q(t) b with phi(0) = phi_0 is
    (K + z M) Phi(z) = q_hat(z) b + M phi_0.

Pinned by tests/test_oracle_initial_rates.py: q_hat against the Laplace
integral of q evaluated by adaptive quadrature, and the whole forward map
against the matrix-exponential solution of the ODE on small grids.
"""
from __future__ import annotations

import numpy as np


def terms(prob, s):
    """(a, lambda) arrays of source s (the constant rate Q_s if the problem gives none)."""
    rt = getattr(prob, "rate_terms", None)
    if rt is None:
        return np.array([float(prob.Q[s])]), np.array([0.0])
    a, lam = rt[s]
    return np.asarray(a, dtype=np.float64), np.asarray(lam, dtype=np.float64)


def q_hat(prob, s, z):
    """Laplace transform of source s's rate at complex z: sum_j a_j / (z + lambda_j)."""
    a, lam = terms(prob, s)
    return complex(np.sum(a / (z + lam)))


def q_time(prob, s, t):
    """Rate of source s at time t >= 0: sum_j a_j exp(-lambda_j t)."""
    a, lam = terms(prob, s)
    return float(np.sum(a * np.exp(-lam * t)))


def initial_state(prob):
    """phi_0 as a flat float64 vector (zeros when the problem has none)."""
    p0 = getattr(prob, "phi0", None)
    if p0 is None:
        return np.zeros(prob.ncell)
    return np.asarray(p0, dtype=np.float64).ravel()
