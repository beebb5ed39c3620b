"""Pins for the FV operator and the forward oracle O1 (contour + direct LU):
the eigen-expansion closed form (exact for homogeneous boxes), Crank-Nicolson
as an independent time-stepper, and structural properties of K and M."""
import numpy as np
import pytest

import workloads as W
from oracle import closed_form, cn, direct, fv


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_K_symmetric_positive_and_rowsums():
    p = W.random_problem(7, 5, 3, variance=1.0, seed=3)
    K, m = fv.assemble(p)
    Kd = K.toarray()
    assert np.allclose(Kd, Kd.T, rtol=0, atol=1e-20)
    ev = np.linalg.eigvalsh(Kd)
    assert ev.min() > 0            # Dirichlet lateral faces make K SPD
    # K 1 = Dirichlet boundary transmissibilities only (interior fluxes cancel)
    f = fv.face_transmissibilities(p.kappa, p.dx, p.dy, p.dz, p.bc)
    bsum = np.zeros((p.nz, p.ny, p.nx))
    bsum[:, :, 0] += f["bx0"]; bsum[:, :, -1] += f["bx1"]
    bsum[:, 0, :] += f["by0"]; bsum[:, -1, :] += f["by1"]
    bsum[0, :, :] += f["bz0"]; bsum[-1, :, :] += f["bz1"]
    assert np.allclose(K @ np.ones(p.ncell), bsum.ravel(), rtol=1e-12, atol=1e-13 * K.diagonal().max())
    assert np.all(m > 0) and np.isclose(m.sum(), (p.Ss * p.dx * p.dy * p.dz).sum())


def test_harmonic_face_series_flux():
    # two cells in series: the face conductance is the harmonic mean
    p = W.random_problem(2, 1, 1, variance=0.0, seed=0, ns=1, nr=1)
    p.kappa = np.array([[[1e-4, 4e-4]]])
    f = fv.face_transmissibilities(p.kappa, p.dx, p.dy, p.dz, p.bc)
    assert np.isclose(f["tx"][0, 0, 0], p.dy * 1.0 / p.dx * 2 * 1e-4 * 4e-4 / 5e-4)


@pytest.mark.parametrize("n", [16, 20])
def test_direct_matches_closed_form_2d(n):
    p = W.config1(n=n, Nz=24)
    h_o1 = direct.forward(p)
    h_o2 = closed_form.heads(p)
    assert _rel(h_o1, h_o2) < 1e-11


def test_config1_closed_form_nz16():
    """Config 1 at full size (64x64, N_z = 16): O1 vs the exact expansion."""
    p = W.config1()
    h1 = direct.forward(p)
    h2 = closed_form.heads(p)
    for it in range(len(p.times)):
        assert _rel(h1[:, :, it], h2[:, :, it]) < 1e-8
    assert np.all(h2 > 0)                     # injection raises the head
    assert np.all(np.diff(h2, axis=2) >= -1e-14 * h2.max())   # non-decreasing in time


def test_direct_matches_closed_form_3d_neumann_top_bottom():
    p = W.random_problem(8, 6, 4, variance=0.0, seed=1, ns=2, nr=3, nt=3, Nz=24)
    h1 = direct.forward(p)
    h2 = closed_form.heads(p)
    assert _rel(h1, h2) < 1e-11


def test_closed_form_nz_convergence():
    """Quadrature error falls with N_z at about the paper's rate."""
    p = W.config1(n=16)
    exact = closed_form.heads(p)
    errs = []
    for Nz in (8, 12, 16):
        p.Nz = Nz
        errs.append(_rel(direct.forward(p), exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8


def test_direct_vs_crank_nicolson_heterogeneous():
    p = W.random_problem(12, 10, 1, variance=1.5, seed=4, ns=1, nr=3, nt=3, Nz=24,
                         t_range=(50.0, 2e3))
    h1 = direct.forward(p)
    h3 = cn.heads(p, steps_per_interval=300)
    assert _rel(h3, h1) < 1e-6


def test_fields_and_superposition():
    p = W.random_problem(9, 9, 1, variance=1.0, seed=6, ns=2, nr=2, nt=2)
    h, F = direct.forward(p, return_fields=True)
    assert np.allclose(F[:, :, p.rec_cells].transpose(0, 2, 1), h, rtol=1e-13, atol=0)
    # linear in Q
    p2 = W.random_problem(9, 9, 1, variance=1.0, seed=6, ns=2, nr=2, nt=2)
    p2.Q = 2.0 * p.Q
    assert np.allclose(direct.forward(p2), 2.0 * h, rtol=1e-12, atol=0)
