"""Pins for the linearised water-table boundary in the oracle (Sec. 2.1: no flux,
and the boundary term (S_y d phi/dt, psi) of the weak form, which adds S_y times
the face area to the storage of the cells on that face).

* In a 2D aquifer (one layer) a water table on the top face is the same as
  storativity Ss + S_y / dz: the closed form of that problem must agree.
* With no-flux faces everywhere else and a constant rate from phi = 0, the
  stored volume sum_c (Ss_c V + S_y,c A_top) phi_c(t) equals the pumped volume
  Q t (the weights computed here from the inputs, not from the oracle's M).
* The adjoint's log-Ss derivative covers Ss V only: central differences of O1.
* Crank-Nicolson (O3) with the same M agrees with O1."""
import copy

import numpy as np

import workloads as W
from oracle import adjoint, closed_form, cn, direct, fv


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_2d_water_table_is_added_storativity():
    p = W.config1(n=24, Nz=24)
    wt = W.with_water_table(p, face=5, sy=0.05)
    eq = copy.copy(p)
    eq.Ss = p.Ss + 0.05 / p.dz
    h_wt = direct.forward(wt)
    assert _rel(h_wt, direct.forward(eq)) < 1e-12
    assert _rel(h_wt, closed_form.heads(eq)) < 1e-8
    # and the water table changes the answer (Sy / dz is far above Ss)
    assert _rel(h_wt, direct.forward(p)) > 0.1


def test_stored_volume_equals_pumped_volume_3d():
    p = W.random_problem(10, 8, 5, variance=1.0, seed=3, ns=1, nr=2, nt=3, Nz=24, ss_variance=0.25,
                         bc=(1, 1, 1, 1, 1, 1))
    p = W.with_water_table(p, face=5, sy=0.1, seed=3, variance=0.3)
    _, F = direct.forward(p, return_fields=True)
    vol = p.dx * p.dy * p.dz
    w = (p.Ss.ravel() * vol).copy()
    top = np.zeros((p.nz, p.ny, p.nx))
    top[-1] = 1.0
    w += p.Sy * top.ravel() * (p.dx * p.dy)
    for it, t in enumerate(p.times):
        stored = float(np.dot(w, F[0, it]))
        assert abs(stored - p.Q[0] * t) <= 1e-8 * p.Q[0] * t


def test_adjoint_log_ss_derivative_with_water_table_vs_finite_differences():
    p = W.random_problem(6, 5, 3, variance=1.0, seed=5, ns=1, nr=2, nt=2, Nz=24, ss_variance=0.25)
    p = W.with_water_table(p, face=5, sy=0.05, seed=5, variance=0.3)
    J = adjoint.jacobian(p)
    top = [c for c in range(p.ncell) if c // (p.nx * p.ny) == p.nz - 1][:4] + [3, 40]
    for which in (0, 1):
        fd = adjoint.fd_jacobian(p, top, which, delta=1e-3)
        an = J[:, :, :, which, :][..., top]
        assert np.linalg.norm(an - fd) / np.linalg.norm(fd) < 1e-6, which


def test_crank_nicolson_with_water_table_matches_o1():
    p = W.random_problem(12, 10, 4, variance=1.0, seed=6, ns=1, nr=3, nt=3, Nz=24)
    p = W.with_water_table(p, face=5, sy=0.1)
    assert _rel(direct.forward(p), cn.heads(p, steps_per_interval=300)) < 1e-6


def test_assembly_adds_face_area_times_sy_on_the_water_table_face_only():
    p = W.random_problem(5, 4, 3, variance=0.5, seed=7, ns=1, nr=1, nt=1)
    wt = W.with_water_table(p, face=4, sy=0.3)          # bottom face
    _, m0 = fv.assemble(p)
    _, m1 = fv.assemble(wt)
    d = (m1 - m0).reshape(p.nz, p.ny, p.nx)
    assert np.allclose(d[0], 0.3 * p.dx * p.dy, rtol=1e-14)
    assert np.all(d[1:] == 0.0)
