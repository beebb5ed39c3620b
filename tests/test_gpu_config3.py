"""Config-3-style adjoint check (3D log-normal kappa and Ss, sources on the
mid layer, receivers on three layers): GPU Jacobian against the FP64 oracle
Jacobian and against central finite differences of the GPU forward solve at
random cells, on a reduced grid."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint

pytestmark = pytest.mark.gpu


def test_config3_reduced_jacobian_vs_oracle_and_fd():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    p = W.config3(nxy=16, nz=8, n_src_side=2, n_rec_side=2, rec_layers=[2, 5], nt=3)
    eng = Engine(0)
    eng.load_problem(p, tol=1e-12)
    ns, nr, nt = len(p.src_cells), len(p.rec_cells), len(p.times)
    J = torch.zeros((ns, nr, nt, 2, p.ncell), dtype=torch.float64, device="cuda")
    eng.adjoint_jacobian(p.times, J)
    torch.cuda.synchronize()
    Jg = J.cpu().numpy()
    ref = adjoint.jacobian(p)
    assert np.linalg.norm(Jg - ref) / np.linalg.norm(ref) < 1e-8
    # central differences of the GPU forward at 8 random cells, both parameters
    rng = np.random.default_rng(64)
    cells = rng.choice(p.ncell, size=8, replace=False)
    delta = 1e-4
    for which in (0, 1):
        fd = np.zeros((ns, nr, nt, len(cells)))
        for ci, c in enumerate(cells):
            hs = []
            for sgn in (1.0, -1.0):
                kap = p.kappa.copy().ravel(); ss = p.Ss.copy().ravel()
                (kap if which == 0 else ss)[c] *= np.exp(sgn * delta)
                eng.setup_grid(kap.reshape(p.kappa.shape), ss.reshape(p.Ss.shape), p.dx, p.dy, p.dz, p.bc)
                eng.set_sources(p.src_cells, p.Q)
                eng.set_receivers(p.rec_cells)
                hs.append(eng.forward(p.times))
            fd[..., ci] = (hs[0] - hs[1]) / (2 * delta)
        an = Jg[:, :, :, which, :][..., cells]
        assert np.abs(an - fd).max() / np.abs(an).max() < 1e-5
    eng.close()
