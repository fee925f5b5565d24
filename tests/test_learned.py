"""Learned correction inside the multigrid cycle (GPU).

The step psi += alpha c takes the alpha that minimises the weighted residual
norm along c, so with the linear fine operator (pg = 0) it never raises the
residual, whatever the network predicts; a solve with it converges to the
plain solve's solution.  With the trained weights shipped in the package, a
scattering-dominated held-out problem needs fewer cycles than plain
multigrid."""
import os

import numpy as np
import pytest

from paper_2301_09991_gb300 import inputs as I

WEIGHTS = os.path.join(os.path.dirname(__file__), "..", "paper_2301_09991_gb300", "weights", "unet_thick.npy")


def _solve(prob, net=None, every=1, rtol=1e-5, max_cycles=3000):
    import torch
    from paper_2301_09991_gb300 import btmg
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    if net is not None:
        gp.set_learned(net, every=every)
    psi = gp.zeros()
    out = gp.solve(psi, rtol=rtol, max_cycles=max_cycles)
    torch.cuda.synchronize()
    return out, psi, (gp.learn_stats() if net is not None else None)


@pytest.mark.gpu
@pytest.mark.parametrize("every", [1, 3])
def test_untrained_net_never_raises_residual_and_converges_to_plain_solution(every):
    import torch
    from paper_2301_09991_gb300 import btmg
    prob = I.checkerboard(n=48, ny=40, n_polar=8, n_azim=16, blocks=4, seed=11, c=0.95, length=5.0)
    plain, p0, _ = _solve(prob)
    net = btmg.UNet(in_channels=btmg.LEARN_FEATURES, seed=3)  # random weights: a poor predictor
    learn, p1, (steps, factor, alpha, fallbacks) = _solve(prob, net, every=every)
    diff = float(torch.linalg.norm(p1 - p0) / torch.linalg.norm(p0))
    print("plain %d cycles, learned(every %d) %d cycles, %d steps, mean factor %.4f, solution diff %.1e"
          % (plain["cycles"], every, learn["cycles"], steps, factor, diff))
    # 1e-5 sits at the FP32 rounding floor of this problem: the returned
    # psi's residual may land just above it
    assert plain["status"] == btmg.OK
    assert learn["status"] in (btmg.OK, btmg.ERR_NOT_CONVERGED) and learn["rel_resid"] <= 1.5e-5
    assert steps == (learn["cycles"] + every - 1) // every
    assert 0.0 < factor <= 1.0 + 1e-6
    assert diff < 5e-5


@pytest.mark.gpu
def test_learned_mg_cycle_and_detach():
    import torch
    from paper_2301_09991_gb300 import btmg
    prob = I.checkerboard(n=40, n_polar=8, n_azim=8, blocks=4, seed=12, c=0.9, length=3.0)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    net = btmg.UNet(in_channels=btmg.LEARN_FEATURES, seed=4)
    gp.set_learned(net, every=2)
    psi = gp.zeros()
    for _ in range(5):
        gp.mg_cycle(psi)
    steps, factor = gp.learn_stats()[:2]
    assert steps == 3 and 0.0 < factor <= 1.0 + 1e-6
    gp.set_learned(None)
    q = psi.clone()
    gp.mg_cycle(q)
    assert gp.learn_stats()[0] == 0
    assert torch.isfinite(q).all()


@pytest.mark.gpu
def test_trained_net_gains_over_plain_multigrid():
    """Held-out problem of the training class (checkerboard, side 20 mean free
    paths of the thickest block, c = 0.99): fewer cycles to 1e-5 than plain
    multigrid, and the same solution."""
    import torch
    from paper_2301_09991_gb300 import btmg
    from paper_2301_09991_gb300 import learned as LN
    if not os.path.exists(WEIGHTS):
        pytest.fail("trained weights missing: " + WEIGHTS)
    net = LN.load_net(WEIGHTS)
    prob = LN.training_problem(5004, n=64, c=0.99, length=20.0)
    plain, p0, _ = _solve(prob)
    learn, p1, (steps, factor, alpha, fallbacks) = _solve(prob, net, every=1)
    diff = float(torch.linalg.norm(p1 - p0) / torch.linalg.norm(p0))
    print("plain %d cycles, learned %d cycles (mean factor %.3f), diff %.1e"
          % (plain["cycles"], learn["cycles"], factor, diff))
    # 1e-5 is at the FP32 rounding floor of this problem: the returned psi's
    # residual may land just above it
    assert learn["status"] in (btmg.OK, btmg.ERR_NOT_CONVERGED) and learn["rel_resid"] <= 1.5e-5
    assert learn["cycles"] < 0.8 * plain["cycles"]
    assert diff < 5e-5
