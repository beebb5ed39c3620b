"""Pins for the oracle's non-zero initial state, exponential-sum pumping rates
(Sec. 2.1-2.2, Sec. 3's right-hand sides [b, M phi_0]), the FOM residual
|eta_k| and the quadrature-weighted stopping rule (Sec. 3.1, Proposition 1).

Each pin compares against something other than the code it checks: the
Laplace integral by adaptive quadrature, the matrix exponential of the ODE
(an augmented linear system, so no inverse of A - lambda I is needed), the
eigen-expansion closed form, Crank-Nicolson, and true residuals computed
from K and M directly."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla

import workloads as W
from oracle import closed_form, cn, contour, direct, fgmres_sh, fv, source


def _prob(nx, ny, variance, seed, ns=2, nr=3, nt=4, Nz=24, bc=None):
    p = W.random_problem(nx, ny, 1, variance=variance, seed=seed, ns=ns, nr=nr, nt=nt, Nz=Nz, bc=bc,
                         t_range=(20.0, 5e3))
    return W.with_initial_state_and_rates(p, seed=seed)


def _expm_heads(p):
    """h[s][r][t] of M phi' + K phi = q_s(t) e_s, phi(0) = phi_0, by the matrix exponential of
    the system augmented with one state u_j' = -lambda_j u_j per rate term (u_j(0) = 1)."""
    K, m = fv.assemble(p)
    A = (K.toarray()) / m[:, None]                     # M^{-1} K
    N = p.ncell
    phi0 = source.initial_state(p)
    h = np.zeros((len(p.src_cells), len(p.rec_cells), len(p.times)))
    for s in range(len(p.src_cells)):
        a, lam = source.terms(p, s)
        J = len(a)
        B = np.zeros((N + J, N + J))
        B[:N, :N] = -A
        for j in range(J):
            B[p.src_cells[s], N + j] = a[j] / m[p.src_cells[s]]
            B[N + j, N + j] = -lam[j]
        x0 = np.concatenate([phi0, np.ones(J)])
        for it, t in enumerate(p.times):
            x = sla.expm(B * t) @ x0
            h[s, :, it] = x[p.rec_cells]
    return h


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_q_hat_is_the_laplace_integral_of_q():
    p = _prob(8, 8, 1.0, seed=1)
    for s in range(2):
        for z in (3e-3, 0.05 + 0.02j, 1e-2 - 4e-3j, 0.2 + 1.0j):
            re = si.quad(lambda t: (np.exp(-z * t) * source.q_time(p, s, t)).real, 0, np.inf, limit=400,
                         epsabs=0, epsrel=1e-11)[0]
            im = si.quad(lambda t: (np.exp(-z * t) * source.q_time(p, s, t)).imag, 0, np.inf, limit=400,
                         epsabs=0, epsrel=1e-11)[0]
            ref = complex(re, im)
            assert abs(source.q_hat(p, s, z) - ref) <= 1e-8 * abs(ref)


def test_constant_rate_is_the_one_term_sum():
    p = W.random_problem(8, 8, 1, seed=2, ns=1, nr=1, nt=1)
    assert source.q_hat(p, 0, 0.3 + 0.1j) == pytest.approx(p.Q[0] / (0.3 + 0.1j), rel=1e-15)
    assert np.all(source.initial_state(p) == 0.0)


@pytest.mark.parametrize("bc", [None, (0, 1, 1, 0, 1, 1)])
def test_o1_matches_matrix_exponential(bc):
    """Heterogeneous 7 x 6 grid, Dirichlet all round or mixed Dirichlet/Neumann faces."""
    p = _prob(7, 6, 1.5, seed=3, bc=bc)
    h = direct.forward(p)
    ref = _expm_heads(p)
    assert _rel(h, ref) < 1e-9


def test_closed_form_with_initial_state_and_rates_matches_expm():
    p = W.random_problem(7, 6, 1, variance=0.0, seed=4, ns=2, nr=3, nt=4, t_range=(20.0, 5e3))
    p = W.with_initial_state_and_rates(p, seed=4)
    assert _rel(closed_form.heads(p), _expm_heads(p)) < 1e-10


def test_closed_form_initial_state_alone_is_a_decaying_mode():
    """phi_0 = one eigenvector of M^{-1} K and no pumping: phi(t) = e^{-mu t} phi_0."""
    p = W.random_problem(9, 7, 1, variance=0.0, seed=5, ns=1, nr=4, nt=3)
    K, m = fv.assemble(p)
    A = K.toarray() / m[:, None]
    mu, V = np.linalg.eigh(K.toarray() / m[0])       # homogeneous: M = m I
    v = V[:, 3]
    p.phi0 = v.copy()
    p.rate_terms = [(np.array([0.0]), np.array([0.0]))]
    h = closed_form.heads(p)
    for it, t in enumerate(p.times):
        assert np.allclose(h[0, :, it], np.exp(-mu[3] * t) * v[p.rec_cells], rtol=1e-10, atol=1e-14)
    assert np.allclose(A @ v, mu[3] * v)


def test_o1_with_initial_state_and_rates_matches_closed_form():
    p = W.config1(n=32, Nz=24)
    p = W.with_initial_state_and_rates(p, seed=6)
    assert _rel(direct.forward(p), closed_form.heads(p)) < 1e-8


def test_o1_matches_crank_nicolson_with_initial_state_and_rates():
    p = _prob(16, 12, 1.5, seed=7, nt=3)
    assert _rel(direct.forward(p), cn.heads(p, steps_per_interval=300)) < 1e-6


def _krylov_setup(n=16, seed=8, t=300.0, Nz=20):
    p = W.random_problem(n, n, 1, variance=1.5, seed=seed, ns=1, nr=1, nt=1, Nz=Nz)
    K, m = fv.assemble(p)
    b = fv.rhs(p, 0)
    z, _ = contour.nodes_weights(t, Nz)
    return p, K, m, b, z


@pytest.mark.parametrize("it", [4, 9, 15])
def test_fom_eta_equals_the_true_residual(it):
    """Proposition 1's proof: b - (K + z_k M) x_k^FOM = -eta_k v_{m+1}, so ||r_k|| = |eta_k| beta."""
    p, K, m, b, z = _krylov_setup()
    taus = contour.tau_schedule(z, "flexible", it)
    X, nit, conv, pres = fgmres_sh.solve(K, m, b, z, taus, tol=1e-300, maxit=it, variant="fom",
                                         return_residuals=True)
    assert nit == it and np.sum(conv < 0) >= len(z) - 1   # only a shift equal to tau_1 stops early
    beta = np.linalg.norm(b)
    for k, zk in enumerate(z):
        r = b - (K @ X[k] + zk * m * X[k])
        assert abs(np.linalg.norm(r) / beta - pres[k]) <= 1e-7 * pres[k] + 1e-12


def test_gmres_residual_is_at_most_fom_residual():
    """The minimal-residual coefficients never do worse than the Petrov-Galerkin ones."""
    p, K, m, b, z = _krylov_setup(seed=9)
    taus = contour.tau_schedule(z, "flexible", 10)
    _, _, _, rg = fgmres_sh.solve(K, m, b, z, taus, tol=1e-300, maxit=10, return_residuals=True)
    _, _, _, rf = fgmres_sh.solve(K, m, b, z, taus, tol=1e-300, maxit=10, variant="fom", return_residuals=True)
    assert np.all(rg <= rf * (1 + 1e-9) + 1e-13)


@pytest.mark.parametrize("variant", ["gmres", "fom"])
def test_quadrature_stop_bounds_the_weighted_true_residual(variant):
    p = W.random_problem(16, 16, 1, variance=1.5, seed=10, ns=1, nr=1, nt=3, Nz=16)
    K, m = fv.assemble(p)
    b = fv.rhs(p, 0) / p.Q[0]
    zs, ws, tid = [], [], []
    for it, t in enumerate(p.times):
        z, w = contour.nodes_weights(t, p.Nz)
        zs.append(z)
        ws.append(np.abs(w * np.array([source.q_hat(p, 0, zk) for zk in z])))
        tid += [it] * len(z)
    zs, ws, tid = np.concatenate(zs), np.concatenate(ws), np.array(tid)
    taus = contour.tau_schedule(zs, "flexible", 300)
    tol = 1e-8
    X, nit, conv = fgmres_sh.solve(K, m, b, zs, taus, tol=tol, maxit=300, variant=variant, stop="quadrature",
                                   weights=ws, time_of=tid)
    assert np.all(conv > 0)
    for it in range(len(p.times)):
        sel = np.where(tid == it)[0]
        assert len(set(conv[sel])) == 1            # the shifts of a time stop together
        tr = np.array([np.linalg.norm(b - (K @ X[k] + zs[k] * m * X[k])) for k in sel])
        assert np.sum(ws[sel] * tr) <= tol * np.sum(ws[sel]) * 1.001
    _, nit_shift, _ = fgmres_sh.solve(K, m, b, zs, taus, tol=tol, maxit=300, variant=variant)
    assert nit <= nit_shift
