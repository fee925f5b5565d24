"""Failure detection without a GPU fault: a bounded wait that nothing
releases gives up, the host reads BTMG_ERR_TIMEOUT, and the context stays
usable (a residual evaluation afterwards matches the oracle)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    assert btmg.wait_selftest(polls=2000) == btmg.ERR_TIMEOUT
    assert btmg.wait_selftest(polls=1) == btmg.ERR_TIMEOUT
    prob = I.checkerboard(n=40, ny=24, n_polar=4, n_azim=8, blocks=4, seed=21)
    gp = btmg.Problem(prob, dtype=btmg.F64, pg=1)
    psi = I.random_field(gp.shape, seed=22)
    r = gp.apply_operator(torch.tensor(psi, device="cuda")).cpu().numpy()
    ref = O.OracleProblem(prob).apply(psi)
    assert np.linalg.norm(r - ref) / np.linalg.norm(ref) < 1e-12


def test_persistent_queue_wait_times_out_and_context_stays_usable():
    """The persistent batched launch waits, bounded, for a task's previous
    level: with a prerequisite that nothing completes the wait gives up (about
    a second), the host reads BTMG_ERR_TIMEOUT, and a batch solve afterwards
    still matches single-problem cycles."""
    L = btmg.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.btmg_batch_wait_selftest(stream) == btmg.ERR_TIMEOUT
    probs = [I.voronoi(24, 4, 8, 31), I.voronoi(40, 8, 8, 32)]
    b = btmg.Batch(probs, dtype=btmg.F32, pg=0)
    assert b.coarse()[0]
    psis = b.zeros()
    rc, infos = b.solve(psis, rtol=0.0, max_cycles=4, check_every=2)
    for i, prob in enumerate(probs):
        gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, chunks=b.chunks(i)[0])
        psi = gp.zeros()
        for _ in range(infos[i]["cycles"]):
            gp.mg_cycle(psi, want_residual=False)
        torch.cuda.synchronize()
        assert torch.equal(psi, psis[i]), i


def test_selftest_rejects_bad_arguments():
    assert btmg.wait_selftest(polls=0) == btmg.ERR_INVALID_ARG
