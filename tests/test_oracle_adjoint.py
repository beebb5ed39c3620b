"""Pins for the Laplace-domain adjoint Jacobian O4 (Sec. 5.2): central
finite differences of the forward oracle, the parameter-scaling invariant
and the time-scaling invariant."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, direct


@pytest.fixture(scope="module")
def small():
    p = W.random_problem(7, 6, 1, variance=1.0, seed=11, ns=2, nr=2, nt=2, Nz=20,
                         ss_variance=0.3, t_range=(30.0, 600.0))
    return p, adjoint.jacobian(p)


def test_fd_log_kappa(small):
    p, J = small
    cells = [0, 8, 20, 41]
    fd = adjoint.fd_jacobian(p, cells, which=0, delta=1e-4)
    an = J[:, :, :, 0, :][..., cells]
    assert np.abs(an - fd).max() / np.abs(an).max() < 1e-6


def test_fd_log_ss(small):
    p, J = small
    cells = [3, 17, 29]
    fd = adjoint.fd_jacobian(p, cells, which=1, delta=1e-4)
    an = J[:, :, :, 1, :][..., cells]
    assert np.abs(an - fd).max() / np.abs(an).max() < 1e-6


def test_scale_invariant(small):
    """kappa -> a kappa, Ss -> a Ss scales phi by 1/a, so
    sum_c (dh/dlog kappa_c + dh/dlog Ss_c) = -h."""
    p, J = small
    h = direct.forward(p)
    lhs = J.sum(axis=(3, 4))
    assert np.abs(lhs + h).max() / np.abs(h).max() < 1e-9


def test_time_scaling_invariant(small):
    """kappa -> a kappa alone is phi_a(t) = phi(a t) / a, so
    sum_c dh/dlog kappa_c = -h + t dh/dt."""
    p, J = small
    h = direct.forward(p)
    dhdt = adjoint.dh_dt(p)
    lhs = J[:, :, :, 0, :].sum(axis=-1)
    rhs = -h + p.times[None, None, :] * dhdt
    assert np.abs(lhs - rhs).max() / np.abs(h).max() < 1e-9


def test_symmetry_homogeneous_source_receiver_swap():
    """Homogeneous field: swapping source and receiver cells leaves the
    sensitivity map unchanged (reciprocity; Sec. 5.2 figure)."""
    n, c = 13, 6                      # odd grid: cell c is the domain centre
    p = W.config1(n=n, Nz=20)
    p.src_cells = np.array([c * n + c]); p.rec_cells = np.array([c * n + c - 3]); p.times = np.array([200.0])
    J1 = adjoint.jacobian(p)
    q = W.config1(n=n, Nz=20)
    q.src_cells = p.rec_cells.copy(); q.rec_cells = p.src_cells.copy(); q.times = p.times.copy()
    J2 = adjoint.jacobian(q)
    assert np.abs(J1 - J2).max() / np.abs(J1).max() < 1e-12
    # mirror symmetry about the source-receiver axis (row c)
    m = J1[0, 0, 0, 0].reshape(n, n)
    assert np.abs(m[c - 2] - m[c + 2]).max() / np.abs(m).max() < 1e-12


def test_fd_with_exponential_sum_rates():
    """O4 with time-varying rates (qhat in place of Q / z) against central differences of O1."""
    p = W.random_problem(6, 5, 1, variance=1.0, seed=11, ns=2, nr=2, nt=2, Nz=24)
    p = W.with_initial_state_and_rates(p, seed=11, initial=False)
    J = adjoint.jacobian(p)
    cells = [0, 7, 13, 29]
    for which in (0, 1):
        fd = adjoint.fd_jacobian(p, cells, which)
        an = J[:, :, :, which, :][..., cells]
        assert np.linalg.norm(an - fd) / np.linalg.norm(fd) < 1e-6
