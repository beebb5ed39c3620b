"""Config 3 at full size (128x128x32, log-normal kappa and Ss): the adjoint
Jacobian against central finite differences of the GPU forward solve on 64
random cells, both parameters (d h / d log kappa_c and d h / d log Ss_c).

Half the cells are uniform over the grid, half within the source's
neighbourhood, where the sensitivities are large.  Each Jacobian row (source,
receiver, time) is compared on the sampled cells relative to its largest
entry over all cells: far from the wells the entries are close to zero while
the finite differences carry the solver's noise, so a per-entry relative error
would measure noise.  The step delta = 2e-3 (in log kappa, log Ss) balances
the central difference's truncation error (about delta^2 / 6 of the entry)
against that noise (about 1e-10 |h| / delta); with delta = 1e-4 the log Ss rows,
which are small next to |h|, were noise-limited at 1.4e-4 of their scale."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_config3_full_size_jacobian_vs_finite_differences_on_64_cells():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    p = W.config3()
    p.src_cells = p.src_cells[5:6]          # one source (FD needs two forward solves per cell)
    p.Q = p.Q[5:6]
    p.times = p.times[[4]]
    eng = Engine(0)
    eng.load_problem(p, tol=1e-12, maxit=120)
    ns, nr, nt = 1, len(p.rec_cells), len(p.times)
    J = torch.zeros((ns, nr, nt, 2, p.ncell), dtype=torch.float64, device="cuda")
    eng.adjoint_jacobian(p.times, J)
    torch.cuda.synchronize()
    st = eng.last_stats
    assert st["n_converged"] == st["n_shift_solves"]
    scale = J.abs().amax(dim=-1).cpu().numpy()          # [ns][nr][nt][2]: largest entry of each row
    rng = np.random.default_rng(64)
    nx = ny = 128
    nz = 32
    sc = int(p.src_cells[0])
    i0, j0, k0 = sc % nx, (sc // nx) % ny, sc // (nx * ny)
    near = [int(((k0 + rng.integers(-3, 4)) * ny + j0 + rng.integers(-16, 17)) * nx + i0 + rng.integers(-16, 17))
            for _ in range(32)]
    far = [int(c) for c in rng.choice(nx * ny * nz, size=32, replace=False)]
    cells = near + far
    delta = 2e-3
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
        err = np.abs(an - fd) / scale[..., which][..., None]
        assert err.max() < 1e-5, (which, err.max())
        # the near-source cells carry real sensitivity: not a comparison of zeros
        assert np.abs(an[..., :32]).max() > 1e-3 * scale[..., which].max()
    eng.close()
