"""GPU parity of the adjoint path: Jacobian (Sec. 5.2) against the FP64
oracle O4 and central finite differences, the vector-Jacobian product, and
the autograd Function."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, direct

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def Engine():
    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    return Engine


def _jac(Engine, p, **kw):
    import torch
    eng = Engine(0)
    eng.load_problem(p, **kw)
    J = torch.zeros((len(p.src_cells), len(p.rec_cells), len(p.times), 2, p.ncell), dtype=torch.float64,
                    device="cuda")
    eng.adjoint_jacobian(p.times, J)
    torch.cuda.synchronize()
    st = eng.last_stats
    eng.close()
    return J.cpu().numpy(), st


@pytest.mark.parametrize("shape", [(10, 8, 1), (12, 12, 1), (6, 6, 4)])
def test_jacobian_vs_oracle(Engine, shape):
    nx, ny, nz = shape
    p = W.random_problem(nx, ny, nz, variance=1.0, seed=nx + nz, ns=2, nr=3, nt=2, Nz=16, tol=1e-12,
                         ss_variance=0.3, t_range=(30.0, 600.0))
    J, st = _jac(Engine, p)
    ref = adjoint.jacobian(p)
    assert _rel(J, ref) < 1e-8
    assert st["n_converged"] == st["n_shift_solves"]


def test_jacobian_vs_finite_differences(Engine):
    p = W.random_problem(9, 7, 1, variance=1.0, seed=5, ns=1, nr=2, nt=2, Nz=16, tol=1e-12, ss_variance=0.2,
                         t_range=(50.0, 500.0))
    J, _ = _jac(Engine, p)
    cells = [0, 10, 31, 62]
    for which in (0, 1):
        fd = adjoint.fd_jacobian(p, cells, which=which, delta=1e-4)
        an = J[:, :, :, which, :][..., cells]
        assert np.abs(an - fd).max() / np.abs(an).max() < 1e-6


def test_vjp_matches_contracted_jacobian_and_returns_h(Engine):
    import torch
    p = W.random_problem(16, 12, 1, variance=1.5, seed=8, ns=2, nr=3, nt=3, Nz=16, tol=1e-12, groups=2)
    J, _ = _jac(Engine, p)
    rng = np.random.default_rng(0)
    g = rng.standard_normal((2, 3, 3))
    eng = Engine(0)
    eng.load_problem(p)
    gd = torch.tensor(g, device="cuda")
    grad = torch.zeros((2, p.ncell), dtype=torch.float64, device="cuda")
    h = torch.zeros((2, 3, 3), dtype=torch.float64, device="cuda")
    eng.adjoint_vjp(p.times, gd, grad, h)
    torch.cuda.synchronize()
    eng.close()
    ref = np.einsum("srt,srtpc->pc", g, J)
    assert _rel(grad.cpu().numpy(), ref) < 1e-10
    assert _rel(h.cpu().numpy(), direct.forward(p)) < 1e-8


def test_autograd_function(Engine):
    import torch

    from paper_1409_2556_gb300.autograd import measurements
    p = W.random_problem(12, 10, 1, variance=1.0, seed=2, ns=2, nr=2, nt=2, Nz=16, tol=1e-12, ss_variance=0.2)
    eng = Engine(0)
    eng.set_options(Nz=16, tol=1e-12)
    lk = torch.tensor(np.log(p.kappa), dtype=torch.float64, requires_grad=True)
    ls = torch.tensor(np.log(p.Ss), dtype=torch.float64, requires_grad=True)
    h = measurements(lk, ls, eng, p)
    assert _rel(h.detach().cpu().numpy(), direct.forward(p)) < 1e-8
    w = torch.tensor(np.random.default_rng(1).standard_normal(h.shape), device=h.device)
    (h * w).sum().backward()
    Jref = adjoint.jacobian(p)
    wn = w.cpu().numpy()
    gk = np.einsum("srt,srtc->c", wn, Jref[:, :, :, 0]).reshape(p.kappa.shape)
    gs = np.einsum("srt,srtc->c", wn, Jref[:, :, :, 1]).reshape(p.Ss.shape)
    assert _rel(lk.grad.numpy(), gk) < 1e-8
    assert _rel(ls.grad.numpy(), gs) < 1e-8
    eng.close()
