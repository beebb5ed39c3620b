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
