"""Learned initial guess for the preconditioner solves: tensor-core U-Net
gradients against the CPU oracle, training on multigrid solves produced by
the library, and use inside the forward solver (FP64 true residual judges)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as G
    G.build()
    from paper_1409_2556_gb300 import Engine, learned
    return Engine, learned


def test_network_gradient_matches_cpu_oracle(mods):
    import torch

    from oracle import unet as U
    _, learned = mods
    net = learned.UNet(0, seed=3)
    theta = net.get_params().astype(np.float64)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 16, 24, 5)).astype(np.float32)
    t = rng.standard_normal((2, 16, 24, 2)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    td = torch.tensor(t, device="cuda")
    out = net.forward(xd).cpu().numpy()
    loss_g, grad_g = net.grad(xd, td)
    loss_c, grad_c, out_c = U.loss_and_grad(theta, x, t)
    assert np.linalg.norm(out - out_c) / np.linalg.norm(out_c) < 3e-2      # bf16 activations
    assert abs(loss_g - loss_c) / loss_c < 2e-2
    cos = grad_g @ grad_c / (np.linalg.norm(grad_g) * np.linalg.norm(grad_c))
    assert cos > 0.995
    assert np.linalg.norm(grad_g - grad_c) / np.linalg.norm(grad_c) < 0.1
    net.close()


def test_training_lowers_loss_and_solver_stays_exact(mods):
    import torch

    from oracle import direct
    Engine, learned = mods
    rng = np.random.default_rng(7)
    xs, ys = [], []
    for prob in learned.training_fields(range(4)):
        eng = Engine(0)
        eng.setup_grid(prob.kappa, prob.Ss, prob.dx, prob.dy, prob.dz, prob.bc)
        x, y = learned.make_pairs(eng, prob, 512, rng, cycles=30)
        xs.append(x); ys.append(y)
        eng.close()
    pairs = (torch.cat(xs), torch.cat(ys))
    net = learned.UNet(0, seed=11)
    hist = learned.train(net, pairs, steps=800, batch=32, lr=2e-3, rng=rng)
    assert np.mean(hist[-50:]) < 0.5 * np.mean(hist[:20])
    # unseen field: the solver with the learned guess still meets the FP64 true residual and the oracle
    p = W.random_problem(64, 64, 1, variance=1.5, seed=77, ns=2, nr=3, nt=3, Nz=16, tol=1e-11)
    res = {}
    for pc in (0, 1):
        eng = Engine(0)
        eng.load_problem(p, precond=pc)
        if pc:
            eng.lib.lt_set_learned_preconditioner(eng.h, net.h)
        h = eng.forward(p.times)
        res[pc] = (h, eng.last_stats)
        eng.close()
    ref = direct.forward(p)
    for pc in (0, 1):
        h, st = res[pc]
        assert np.linalg.norm(h - ref) / np.linalg.norm(ref) < 1e-8
        assert st["n_converged"] == st["n_shift_solves"]
    kept = res[1][1]["work"][14]
    print("learned guess kept in", kept, "rounds; ms without/with:", res[0][1]["ms_total"], res[1][1]["ms_total"])
    # what the trained network gains: the solver keeps a guess only when it removes at least 5% of the
    # residual norm of a preconditioner solve's first round, and on the unseen field it keeps some
    assert kept >= 1
    net.close()
