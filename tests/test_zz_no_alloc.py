"""lt_forward_noalloc: the forward solve for callers that cannot let the
library allocate device memory (their device memory belongs to their own
pool allocator, or they cannot afford the device synchronisation of
cudaMalloc/cudaFree).  Its buffers come from a fixed static region inside the
library.  Checked through the C ABI against lt_forward on two calls in a row;
this file is collected last so that a failure here leaves the other tests'
results intact."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL_H = 1e-8


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_forward_on_two_calls():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    p = W.random_problem(24, 24, 1, variance=1.0, seed=21, ns=2, nr=3, nt=2, Nz=16, tol=1e-11)
    eng = Engine(0)
    eng.load_problem(p, maxit=64)
    shape = (2, 3, 2)
    ref = torch.zeros(shape, dtype=torch.float64, device="cuda")
    eng.forward(p.times, out=ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    outs = []
    for _ in range(2):
        out = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        eng.forward_noalloc(p.times, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
        assert eng.last_stats["n_converged"] == eng.last_stats["n_shift_solves"] == 2 * 2 * 8
    for o in outs:
        assert np.all(np.isfinite(o))
        assert _rel(o, ref) < TOL_H
    # the ordinary entry point still works after the static-region calls
    again = torch.zeros(shape, dtype=torch.float64, device="cuda")
    eng.forward(p.times, out=again)
    torch.cuda.synchronize()
    assert _rel(again.cpu().numpy(), ref) < TOL_H
    eng.close()


def test_noalloc_cluster_path_matches_forward_and_allocates_nothing():
    """64 x 32 splits into the cluster-resident preconditioner solve (its finest-level
    scratch then also comes from the static region); after a warm-up call, a call
    leaves the device's free memory unchanged."""
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine
    p = W.random_problem(64, 32, 1, variance=1.0, seed=22, ns=2, nr=3, nt=2, Nz=16, tol=1e-11)
    eng = Engine(0)
    eng.load_problem(p, maxit=64)
    shape = (2, 3, 2)
    ref = torch.zeros(shape, dtype=torch.float64, device="cuda")
    eng.forward(p.times, out=ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    out = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    eng.forward_noalloc(p.times, out)          # warm-up: loads every kernel module it uses
    torch.cuda.synchronize()
    assert eng.last_stats["work"][15] > 0      # the cluster-resident solve ran
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        out.fill_(float("nan"))
        eng.forward_noalloc(p.times, out)
        torch.cuda.synchronize()
        assert eng.last_stats["work"][15] > 0
        assert eng.last_stats["n_converged"] == eng.last_stats["n_shift_solves"] == 2 * 2 * 8
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert _rel(o, ref) < TOL_H
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    eng.close()


def test_noalloc_rejects_problems_larger_than_its_region():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine, LtError
    p = W.random_problem(128, 128, 1, variance=1.0, seed=3, ns=4, nr=2, nt=3, Nz=16)
    eng = Engine(0)
    eng.load_problem(p)
    out = torch.zeros((4, 2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(LtError) as e:
        eng.forward_noalloc(p.times, out)
    assert e.value.code == -1 and "bytes" in str(e.value)
    eng.close()
