"""Config 3 at full size (128x128x32, log-normal kappa and Ss): the adjoint
Jacobian of one source against central finite differences of the GPU
forward solve at random cells (both parameters)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_config3_full_size_jacobian_vs_finite_differences():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    p = W.config3()
    p.src_cells = p.src_cells[5:6]          # one source (FD needs two forward solves per cell)
    p.Q = p.Q[5:6]
    p.rec_cells = p.rec_cells[16:32]        # the mid-layer receivers
    p.times = p.times[[2, 6]]
    eng = Engine(0)
    eng.load_problem(p, tol=1e-11, maxit=96)
    ns, nr, nt = 1, len(p.rec_cells), len(p.times)
    J = torch.zeros((ns, nr, nt, 2, p.ncell), dtype=torch.float64, device="cuda")
    eng.adjoint_jacobian(p.times, J)
    torch.cuda.synchronize()
    st = eng.last_stats
    assert st["n_converged"] == st["n_shift_solves"]
    # random cells near the source, where the sensitivities are not negligible
    rng = np.random.default_rng(64)
    sc = int(p.src_cells[0])
    nx = ny = 128
    i0, j0, k0 = sc % nx, (sc // nx) % ny, sc // (nx * ny)
    cells = [((k0 + rng.integers(-3, 4)) * ny + j0 + rng.integers(-16, 17)) * nx + i0 + rng.integers(-16, 17)
             for _ in range(12)]
    delta = 1e-4
    Jg = J.cpu().numpy()
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
        assert np.abs(an - fd).max() / np.abs(an).max() < 1e-4, (which, np.abs(an - fd).max(), np.abs(an).max())
    eng.close()
