"""FP64 CPU oracle for the Laplace-transform / shifted-Krylov engine.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; it
is imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  It shares no
code with the CUDA path.

Contents, each following the paper (Bakhos, Saibaba, Kitanidis, "A fast
algorithm for parabolic PDE-based inverse problems based on Laplace
transforms and flexible Krylov solvers"):

* ``fv``          cell-centred finite-volume K, M, b (restating the
                  semi-discrete system of Sec. 2.1, Eq. (2.3)-(2.4)).
* ``contour``     modified Talbot contour, trapezoid nodes and weights,
                  conjugate half-sum (Sec. 2.2, Eq. talbot, quadrature, half).
* ``direct``      O1: contour + sparse direct LU per shifted system.
* ``closed_form`` O2: eigenfunction expansion of the discrete operator for a
                  homogeneous box (exact for the semi-discrete ODE).
* ``cn``          O3: Crank-Nicolson time stepping (the paper's comparison
                  method, Sec. 1 and Sec. 5.3) with a Rannacher start.
* ``fgmres_sh``   Algorithm 1, flexible GMRES/FOM for shifted systems with
                  exact shift-and-invert preconditioners (Sec. 3).
* ``adjoint``     O4: Laplace-domain adjoint Jacobian (Sec. 5.2) and central
                  finite differences.

Parity pinning status is stated in each module header.
"""
