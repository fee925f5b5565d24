"""NaN injection on the host: a NaN in the caller's initial guess ends a
solve with BTMG_ERR_NAN (no hang, no false convergence), in a plain, a
refined and a batched solve (where only the poisoned member fails), and
non-finite or negative materials are rejected when the problem is created."""
import numpy as np
import pytest
import torch

from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu


def _prob():
    return I.checkerboard(n=40, ny=32, n_polar=4, n_azim=8, blocks=4, seed=51, c=0.8)


@pytest.mark.parametrize("pg", [0, 1])
def test_nan_in_initial_guess_ends_solve_with_nan_status(pg):
    gp = btmg.Problem(_prob(), dtype=btmg.F32, pg=pg)
    psi = gp.zeros()
    psi[0, 3, 10, 7] = float("nan")
    out = gp.solve(psi, rtol=1e-5, max_cycles=200)
    assert out["status"] == btmg.ERR_NAN, out
    assert out["cycles"] < 200


def test_nan_in_refined_solve():
    gp = btmg.Problem(_prob(), dtype=btmg.BF16, pg=0)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    psi64[0, 1, 5, 5] = float("nan")
    with pytest.raises(btmg.BtmgError) as e:
        gp.solve_refined(psi64, rtol=1e-8, max_outer=20, inner_cycles=4)
    assert e.value.code == btmg.ERR_NAN


def test_nan_member_of_a_batch_fails_alone():
    probs = [_prob(), I.voronoi(24, 4, 8, 52), I.voronoi(32, 8, 8, 53)]
    b = btmg.Batch(probs, dtype=btmg.F32, pg=0)
    psis = b.zeros()
    psis[1][0, 0, 3, 3] = float("nan")
    rc, infos = b.solve(psis, rtol=1e-5, max_cycles=400)
    assert rc == btmg.ERR_NOT_CONVERGED
    assert infos[1]["status"] == btmg.ERR_NAN
    assert infos[0]["status"] == btmg.OK and infos[2]["status"] == btmg.OK, infos


@pytest.mark.parametrize("field,value", [("sigma_t", np.nan), ("sigma_t", -1.0), ("sigma_s", np.inf),
                                         ("source", np.nan)])
def test_bad_materials_are_rejected(field, value):
    prob = _prob()
    arr = np.array(prob[field], dtype=np.float64)
    arr.reshape(-1)[2] = value
    prob = dict(prob, **{field: arr})
    with pytest.raises(btmg.BtmgError) as e:
        btmg.Problem(prob, dtype=btmg.F32, pg=0)
    assert e.value.code == btmg.ERR_INVALID_ARG
