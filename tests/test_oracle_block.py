"""Pins for the oracle's block flexible GMRES for shifted systems (Algorithm 1 with the sources'
right-hand sides as one block; the block Krylov variant of Sec. 6's future work):

* p = 1 is Algorithm 1: the same iterations, convergence and solutions as oracle/fgmres_sh;
* the block flexible Arnoldi identity (K + z M) U_m = V_{m+1} Hbar(z) holds to rounding;
* the solutions equal the direct LU of every shifted system to the tolerance, and the block
  needs no more outer iterations than the slowest single source."""
import numpy as np
import pytest

import workloads as W
from oracle import block_fgmres, contour, direct, fgmres_sh, fv


def _setup(n=20, ns=4, seed=3, Nz=16, t=300.0):
    p = W.random_problem(n, n, 1, variance=1.5, seed=seed, ns=ns, nr=1, nt=1, Nz=Nz)
    K, m = fv.assemble(p)
    B = np.stack([fv.rhs(p, s) / p.Q[s] for s in range(ns)], 1)
    z, _ = contour.nodes_weights(t, Nz)
    return p, K, m, B, z


def test_block_of_one_is_algorithm1():
    p, K, m, B, z = _setup(ns=1)
    taus = contour.tau_schedule(z, "flexible", 300)
    Xb, itb, convb, _ = block_fgmres.solve(K, m, B, z, taus, tol=1e-10, maxit=300)
    X1, it1, conv1 = fgmres_sh.solve(K, m, B[:, 0], z, taus, tol=1e-10, maxit=300)
    assert itb == it1
    assert np.array_equal(convb[:, 0], conv1)
    assert np.abs(Xb[:, :, 0] - X1).max() <= 1e-10 * np.abs(X1).max()


def test_block_arnoldi_identity():
    p, K, m, B, z = _setup(n=12, ns=3)
    taus = contour.tau_schedule(z, "flexible", 10)
    for zk in z[[0, 4, 7]]:
        assert block_fgmres.arnoldi_identity_error(K, m, B, zk, taus, 8) < 1e-12


def test_block_solutions_match_lu_in_no_more_iterations():
    p, K, m, B, z = _setup()
    taus = contour.tau_schedule(z, "flexible", 300)
    X, it, conv, res = block_fgmres.solve(K, m, B, z, taus, tol=1e-10, maxit=300)
    assert np.all(conv > 0)
    for k, zk in enumerate(z):
        for q in range(B.shape[1]):
            r = B[:, q] - (K @ X[k, :, q] + zk * m * X[k, :, q])
            assert np.linalg.norm(r) / np.linalg.norm(B[:, q]) < 2e-10
    singles = [fgmres_sh.solve(K, m, B[:, q], z, taus, tol=1e-10, maxit=300)[1] for q in range(B.shape[1])]
    assert it <= max(singles)
