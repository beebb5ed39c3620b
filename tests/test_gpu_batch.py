"""Batched forward solves of independent aquifers (lt_forward_batch): each
aquifer's result equals its own lt_forward and the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import direct

pytestmark = pytest.mark.gpu


def test_batch_matches_individual_and_oracle():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    from paper_1409_2556_gb300.batch import forward_batch
    probs = [W.random_problem(48, 48, 1, variance=1.0, seed=1, ns=2, nr=3, nt=3, Nz=16, tol=1e-11, groups=2),
             W.random_problem(64, 32, 1, variance=2.0, seed=2, ns=4, nr=2, nt=2, Nz=24, tol=1e-11),
             W.random_problem(96, 96, 1, variance=0.5, seed=3, ns=1, nr=5, nt=4, Nz=16, tol=1e-11, groups=2),
             W.random_problem(16, 16, 8, variance=1.0, seed=4, ns=2, nr=2, nt=2, Nz=16, tol=1e-11)]
    streams = [torch.cuda.Stream() for _ in probs]
    engs = []
    for p, st in zip(probs, streams):
        e = Engine(0, stream=st)
        e.load_problem(p)
        engs.append(e)
    hs, stats = forward_batch(engs, [p.times for p in probs])
    for e, p, h, st in zip(engs, probs, hs, stats):
        single = e.forward(p.times)
        assert np.linalg.norm(h - single) / np.linalg.norm(single) < 1e-12
        ref = direct.forward(p)
        assert np.linalg.norm(h - ref) / np.linalg.norm(ref) < 1e-8
        assert st["n_converged"] == st["n_shift_solves"]
    for e in engs:
        e.close()


def test_adjoint_batch_matches_oracle_per_aquifer():
    """lt_adjoint_batch over uneven aquifers: the materialised Jacobian of one and the
    vector-Jacobian products of the others equal the discrete adjoint oracle O4 (Sec. 5.2)."""
    import torch

    import __graft_entry__ as G
    G.build()
    from oracle import adjoint
    from paper_1409_2556_gb300 import Engine
    from paper_1409_2556_gb300.batch import adjoint_batch
    probs = [W.random_problem(16, 12, 1, variance=1.0, seed=5, ns=2, nr=3, nt=2, Nz=16, tol=1e-12),
             W.random_problem(24, 16, 1, variance=2.0, seed=6, ns=3, nr=2, nt=3, Nz=16, tol=1e-12, groups=2),
             W.random_problem(8, 8, 4, variance=1.0, seed=7, ns=2, nr=2, nt=2, Nz=16, tol=1e-12, ss_variance=0.25)]
    probs[1] = W.with_initial_state_and_rates(probs[1], seed=6, initial=False)
    engs = []
    for p in probs:
        e = Engine(0, stream=torch.cuda.Stream())
        e.load_problem(p)
        engs.append(e)
    dev = "cuda"
    shape = lambda p: (len(p.src_cells), len(p.rec_cells), len(p.times))
    J0 = torch.zeros(shape(probs[0]) + (2, probs[0].ncell), dtype=torch.float64, device=dev)
    rng = np.random.default_rng(3)
    gs = [None] + [torch.tensor(rng.standard_normal(shape(p)), device=dev) for p in probs[1:]]
    grads = [None] + [torch.zeros((2, p.ncell), dtype=torch.float64, device=dev) for p in probs[1:]]
    hs = [torch.zeros(shape(p), dtype=torch.float64, device=dev) for p in probs]
    stats = adjoint_batch(engs, [p.times for p in probs], J=[J0, None, None], g=gs, grad=grads, h=hs)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        ref = adjoint.jacobian(p)
        if i == 0:
            got = J0.cpu().numpy()
        else:
            got = grads[i].cpu().numpy()
            ref = np.einsum("srt,srtpc->pc", gs[i].cpu().numpy(), ref)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8, i
        h_ref = direct.forward(p)
        assert np.linalg.norm(hs[i].cpu().numpy() - h_ref) / np.linalg.norm(h_ref) < 1e-8
        assert stats[i]["n_converged"] == stats[i]["n_shift_solves"]
    for e in engs:
        e.close()
