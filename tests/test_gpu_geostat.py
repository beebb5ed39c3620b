"""GPU parity of the quasi-linear geostatistical inversion (Sec. 5.1, Algorithm 2) through the C
ABI against the oracle's Algorithm 2 with the dense covariance matrix: one iteration (s_{k+1},
beta, xi, h) on ragged 2D grids, and a few iterations of the full loop.  The GPU forms Q J^T by
FFT on the circulant embedding, which is exact; the bar is 1e-8 relative."""
import numpy as np
import pytest

import workloads as W
from oracle import geostat

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine, inversion
    return Engine, inversion


def _data(p, sigma2, ell, seed):
    rng = np.random.default_rng(seed)
    Q = geostat.exp_covariance(p, sigma2, ell)
    Lq = np.linalg.cholesky(Q + 1e-12 * np.eye(p.ncell))
    s_true = np.log(1e-4) + Lq @ rng.standard_normal(p.ncell)
    h_true, _ = geostat.forward_and_jacobian(p, s_true)
    R = np.full(h_true.size, (1e-3 * np.abs(h_true).max()) ** 2)
    y = h_true + np.sqrt(R) * rng.standard_normal(h_true.size)
    return Q, R, y


@pytest.mark.parametrize("shape", [(24, 20), (32, 16)])
def test_one_iteration_matches_oracle(mods, shape):
    Engine, inversion = mods
    nx, ny = shape
    p = W.random_problem(nx, ny, 1, variance=1.0, seed=61, ns=2, nr=3, nt=2, Nz=16, tol=1e-12)
    sigma2, ell = 0.6, 30.0
    Q, R, y = _data(p, sigma2, ell, 62)
    s_k = np.log(p.kappa.ravel())
    h, J = geostat.forward_and_jacobian(p, s_k)
    s_ref, beta_ref, xi_ref = geostat.gn_step(Q, R, np.ones((p.ncell, 1)), y, s_k, h, J)
    eng = Engine(0)
    eng.load_problem(p)
    s_next, beta, xi, hg = inversion.geostat_step(eng, p.times, y, R, sigma2, ell)
    eng.close()
    assert _rel(hg, h) < 1e-8
    assert _rel(s_next, s_ref) < 1e-8
    assert abs(beta - beta_ref[0]) <= 1e-8 * abs(beta_ref[0])
    assert _rel(xi, xi_ref) < 1e-7


def test_gauss_newton_iterations_match_oracle(mods):
    Engine, inversion = mods
    p = W.random_problem(16, 16, 1, variance=0.0, seed=63, ns=2, nr=4, nt=2, Nz=16, tol=1e-12)
    sigma2, ell = 0.5, 40.0
    _, R, y = _data(p, sigma2, ell, 64)
    s0 = np.full(p.ncell, np.log(1e-4))
    s_ref, hist_ref = geostat.gauss_newton(p, y, R, sigma2, ell, s0, iters=3, tol=0.0)
    eng = Engine(0)
    eng.load_problem(p)
    s, hist = inversion.gauss_newton(eng, p, y, R, sigma2, ell, s0, iters=3, tol=0.0)
    eng.close()
    assert len(hist) == 3
    assert _rel(s, s_ref) < 1e-7
    assert hist[-1]["misfit"] < 0.1 * hist[0]["misfit"]
