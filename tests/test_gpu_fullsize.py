"""Parity at the benchmark's full size and launch configuration (256x256
heterogeneous aquifer, 9 wells, 25 receivers, 12 times, 32 nodes, 3 groups,
bench.SOLVE_OPTS): sampled measurements against the FP64 oracle computed
one by one (one source, two times), and the true residual of every shift."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_config2_full_size_sampled():
    import __graft_entry__ as G
    G.build()
    import bench
    from oracle import direct
    from paper_1409_2556_gb300 import Engine
    prob = bench.workload(0)
    eng = Engine(0)
    eng.load_problem(prob, **bench.SOLVE_OPTS)
    from paper_1409_2556_gb300.autotune import autotune
    autotune(eng, prob, bench.SOLVE_OPTS)          # the configuration bench.py times
    h = eng.forward(prob.times)
    st = eng.last_stats
    eng.close()
    assert st["n_shift_solves"] == 9 * 12 * 16
    assert st["n_converged"] == st["n_shift_solves"]
    assert st["max_true_residual"] <= bench.RESIDUAL_BAR
    s = 4
    tsel = [0, 6, 11]
    ref = direct.forward(prob, sources=[s], times=prob.times[tsel])[0]
    got = h[s][:, tsel]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-8, err
