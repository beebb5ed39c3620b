"""Modified Talbot contour and trapezoid quadrature (Sec. 2.2).

The paper prints the contour family z(theta) = sigma + mu (theta cot theta
+ nu i theta) and states (Sec. 2.3) the convergence rate exp(-c N_z) with
c = log 3.89 for the parameters of its reference on Talbot quadratures
(Trefethen, Weideman & Schmelzer, BIT 2006), where sigma and mu scale with
N_z / t.  That rate is reached by the modified family with a cot(alpha
theta) argument; the parameter set used here is

    z(theta) = (N_z / t) * (-0.6122 + 0.5017 theta cot(0.6407 theta) + 0.2645 i theta)

evaluated at the midpoints theta_k = -pi + (2k - 1) pi / N_z of a uniform
grid of spacing 2 pi / N_z on [-pi, pi].  With f(t) = (1/2 pi i) int e^{zt}
F(z) dz the trapezoid rule gives weights

    w_k = -(i / N_z) e^{z_k t} z'(theta_k),    f(t) ~ sum_k w_k F(z_k),

and for F(conj z) = conj F(z) (real K, M, b) the sum folds onto the
upper-half nodes: f(t) ~ 2 Re sum_{k=1}^{N_z/2} w_k F(z_k) (Eq. half).
The paper prints the weight constant as -i/(2N); the quadrature above (and
the tests against known transforms) fix it at -i/N_z.

Pinned by tests/test_oracle_contour.py: inversion of 1/(z + a) -> e^{-a t}
and 1/z -> 1 with the error falling at the stated rate 3.89^{-N_z}.
"""
from __future__ import annotations

import numpy as np

TALBOT_SIGMA = -0.6122
TALBOT_MU = 0.5017
TALBOT_ALPHA = 0.6407
TALBOT_NU = 0.2645


def theta_nodes(Nz: int, half: bool = True) -> np.ndarray:
    k = np.arange(1, Nz + 1)
    th = -np.pi + (2 * k - 1) * np.pi / Nz
    if half:
        th = th[th > 0]
    return th


def z_of_theta(theta, t, Nz):
    th = np.asarray(theta, dtype=np.float64)
    a = TALBOT_ALPHA * th
    return (Nz / t) * (TALBOT_SIGMA + TALBOT_MU * th / np.tan(a) + 1j * TALBOT_NU * th)


def dz_dtheta(theta, t, Nz):
    th = np.asarray(theta, dtype=np.float64)
    a = TALBOT_ALPHA * th
    s = np.sin(a)
    return (Nz / t) * (TALBOT_MU * (1.0 / np.tan(a) - a / (s * s)) + 1j * TALBOT_NU)


def nodes_weights(t: float, Nz: int, half: bool = True):
    """Shifts z_k and weights w_k = -(i/N_z) e^{z_k t} z'(theta_k).

    half=True returns the N_z/2 nodes with Im z > 0 (use with 2 Re sum);
    half=False returns all N_z nodes (use with the plain sum)."""
    th = theta_nodes(Nz, half)
    z = z_of_theta(th, t, Nz)
    w = -(1j / Nz) * np.exp(z * t) * dz_dtheta(th, t, Nz)
    return z, w


def invert_scalar(Fhat, t: float, Nz: int) -> float:
    """Invert a scalar transform F(z) with F(conj z) = conj F(z)."""
    z, w = nodes_weights(t, Nz, half=True)
    return float(2.0 * np.real(np.sum(w * Fhat(z))))


def tau_schedule(zs: np.ndarray, policy: str = "flexible", maxit: int = 1000):
    """Preconditioner shifts tau_j, j = 1..maxit (Sec. 3, last paragraph).

    'single'   : tau = node with the smallest real part (Sec. 4.1).
    'flexible' : tau_bar1 = smallest real part, tau_bar2 = largest real
                 part; tau_j = tau_bar1 for j = 1, 2, 3 and tau_bar2 for
                 j = 4, 5, repeated.
    """
    zs = np.asarray(zs).ravel()
    t1 = zs[np.argmin(zs.real)]
    t2 = zs[np.argmax(zs.real)]
    if policy == "single":
        return np.full(maxit, t1)
    pat = np.array([t1, t1, t1, t2, t2])
    return np.resize(pat, maxit)
