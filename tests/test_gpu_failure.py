"""Failure detection without a GPU fault: a bounded wait that nothing
releases gives up, the host reads BTMG_ERR_TIMEOUT, and the context stays
usable (a residual evaluation afterwards matches the oracle)."""
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


def test_selftest_rejects_bad_arguments():
    assert btmg.wait_selftest(polls=0) == btmg.ERR_INVALID_ARG
