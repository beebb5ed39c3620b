"""Pins for Algorithm 1 (FGMRES-Sh with exact shift-and-invert
preconditioners): solutions equal direct LU to the tolerance; the flexible
Arnoldi relation holds to rounding; iteration trends the paper reports."""
import numpy as np
import pytest

import workloads as W
from oracle import contour, direct, fgmres_sh, fv


def _setup(n=24, var=1.5, seed=0, t=300.0, Nz=20):
    p = W.random_problem(n, n, 1, variance=var, seed=seed, ns=1, nr=1, nt=1, Nz=Nz)
    K, m = fv.assemble(p)
    b = fv.rhs(p, 0)
    z, w = contour.nodes_weights(t, Nz)
    return p, K, m, b, z


@pytest.mark.parametrize("policy", ["single", "flexible"])
def test_fgmres_sh_matches_direct(policy):
    p, K, m, b, z = _setup()
    taus = contour.tau_schedule(z, policy, 400)
    X, it, conv = fgmres_sh.solve(K, m, b, z, taus, tol=1e-10, maxit=400)
    assert np.all(conv > 0)
    for k, zk in enumerate(z):
        ref = direct.shifted_solve(K, m, zk, b)
        r = b - (K @ X[k] + zk * m * X[k])
        assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-10
        assert np.linalg.norm(X[k] - ref) / np.linalg.norm(ref) < 1e-6


def test_fom_variant_converges():
    p, K, m, b, z = _setup(n=16)
    taus = contour.tau_schedule(z, "flexible", 300)
    X, it, conv = fgmres_sh.solve(K, m, b, z, taus, tol=1e-10, maxit=300, variant="fom")
    for k, zk in enumerate(z):
        r = b - (K @ X[k] + zk * m * X[k])
        assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-9


def test_flexible_arnoldi_identity():
    p, K, m, b, z = _setup(n=12)
    taus = contour.tau_schedule(z, "flexible", 12)
    for zk in z[[0, 5, 9]]:
        assert fgmres_sh.arnoldi_identity_error(K, m, b, zk, taus, 10) < 1e-12


def test_flexible_needs_fewer_iterations_than_single():
    """Sec. 4.2, Tables 1-2: two preconditioner shifts beat one."""
    p, K, m, b, z = _setup(n=32, var=1.6, t=300.0, Nz=40)
    _, it_s, _ = fgmres_sh.solve(K, m, b, z, contour.tau_schedule(z, "single", 500), tol=1e-10, maxit=500)
    _, it_f, _ = fgmres_sh.solve(K, m, b, z, contour.tau_schedule(z, "flexible", 500), tol=1e-10, maxit=500)
    assert it_f < it_s
