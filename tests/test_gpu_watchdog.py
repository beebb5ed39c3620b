"""The bounded device wait of the TMA-staged multigrid tiles.

Every TMA tile load waits on an mbarrier for at most `tma_wait_polls` polls;
when that limit runs out the block raises an error flag, lets the copies in
flight land (a second bounded wait) and returns, and the host reports
LT_ERR_TIMEOUT.  Setting the limit to 0 makes every wait run out at once
without any fault: the copies are ordinary in-bounds copies that complete.
No shifted system may then be reported as converged, and the context must
stay usable.  The tensor-core convolutions of the learned preconditioner wait
on the mbarrier their MMAs complete on in the same bounded way."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_tma_wait_that_runs_out_reports_timeout_and_context_recovers():
    import __graft_entry__ as G
    G.build()
    from oracle import direct
    from paper_1409_2556_gb300 import Engine, LtError
    p = W.random_problem(64, 64, 1, variance=1.0, seed=4, ns=2, nr=3, nt=2, Nz=16, tol=1e-10)
    eng = Engine(0)
    # batched multigrid launches with TMA-staged 2D tiles (64 x 64: level 0 takes the fused TMA tiles)
    eng.load_problem(p, mg_cluster=0, mg_tma=1, tma_wait_polls=0, graphs=0)
    with pytest.raises(LtError) as e:
        eng.forward(p.times)
    assert e.value.code == -5, e.value
    assert eng.last_stats["n_converged"] == 0
    # the same context solves correctly once the wait limit is back to its default
    eng.set_options(tma_wait_polls=1 << 26)
    h = eng.forward(p.times)
    ref = direct.forward(p)
    assert np.linalg.norm(h - ref) / np.linalg.norm(ref) < 1e-8
    assert eng.last_stats["work"][13] > 0      # fused_up tiles ran
    eng.close()


def test_precond_apply_reports_timeout():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine, LtError
    p = W.random_problem(64, 64, 1, variance=1.0, seed=5, ns=1, nr=1, nt=1, Nz=16)
    eng = Engine(0)
    eng.load_problem(p, mg_tma=1, tma_wait_polls=0)
    r = torch.randn(2, p.ncell, 2, dtype=torch.float32, device="cuda")
    e = torch.zeros_like(r)
    tau = np.array([[1e-3, 0.0], [2e-3, 1e-3]])
    import ctypes as C
    with pytest.raises(LtError) as err:
        eng._check(eng.lib.lt_precond_apply(eng.h, 2, tau.ctypes.data_as(C.c_void_p), C.c_void_p(r.data_ptr()),
                                            C.c_void_p(e.data_ptr()), 2), "lt_precond_apply")
    assert err.value.code == -5
    eng.set_options(tma_wait_polls=1 << 26)
    eng._check(eng.lib.lt_precond_apply(eng.h, 2, tau.ctypes.data_as(C.c_void_p), C.c_void_p(r.data_ptr()),
                                        C.c_void_p(e.data_ptr()), 2), "lt_precond_apply")
    torch.cuda.synchronize()
    assert torch.isfinite(e).all()
    eng.close()


def test_tensor_core_wait_that_runs_out_reports_timeout_and_network_recovers():
    """Poll limit 0: every convolution's wait runs out at once (the MMAs are ordinary and complete),
    the block waits for them within its second bound, frees its tensor memory and returns; the call
    reports LT_ERR_TIMEOUT, and with the default limit the same network gives its earlier output."""
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import LtError, learned
    net = learned.UNet(0, seed=3)
    x = torch.randn(3, 32, 40, 5, device="cuda")
    ref = net.forward(x)
    net.set_wait_polls(0)
    with pytest.raises(LtError) as e:
        net.forward(x)
    assert e.value.code == -5, e.value
    net.set_wait_polls(1 << 22)
    out = net.forward(x)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    net.close()
