"""Mixed precision: psi stored in BF16 / FP16 with FP32 accumulation, and
FP64 iterative refinement on the GPU.  Checked against the FP64 oracle; the
error against the oracle is asserted (and reported) per group."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu

LOWP = [(btmg.BF16, torch.bfloat16), (btmg.F16, torch.float16)]


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("code,tdt", LOWP)
def test_lowp_storage_operator_parity(code, tdt):
    """Inputs exactly representable in the storage type; FP32 arithmetic."""
    prob = I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=11)
    gp = btmg.Problem(prob, dtype=code)
    op = O.OracleProblem(prob)
    psi = torch.tensor(I.random_field(gp.shape, seed=6), dtype=tdt, device="cuda")
    r = gp.apply_operator(psi).double().cpu().numpy()
    assert rel(r, op.apply(psi.double().cpu().numpy())) < 1e-6


@pytest.mark.parametrize("code,tdt", LOWP)
def test_lowp_cycle_within_storage_precision(code, tdt):
    prob = I.checkerboard(n=40, n_polar=8, n_azim=8, blocks=4, seed=3)
    gp = btmg.Problem(prob, dtype=code, pg=0)
    op = O.OracleProblem(prob, pg=0)
    psi = gp.zeros()
    gp.mg_cycle(psi)
    ref, _, _ = op.mg_cycle(op.zeros())
    eps = 2.0 ** -8 if code == btmg.BF16 else 2.0 ** -11
    assert rel(psi.double().cpu().numpy(), ref) < 4 * eps


@pytest.mark.parametrize("code", [btmg.BF16, btmg.F16, btmg.F32])
def test_refined_multigroup_matches_fp64_oracle_per_group(code):
    prob = I.multigroup(n=24, n_polar=4, n_azim=8, G=3, blocks=3, seed=6)
    gp = btmg.Problem(prob, dtype=code, pg=0)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    out = gp.solve_refined(psi64, rtol=1e-10, max_outer=80, inner_cycles=4)
    assert out["status"] == btmg.OK and out["rel_resid"] <= 1e-10, out
    op = O.OracleProblem(prob, pg=0)
    ref, n, rr, _ = op.solve(rtol=1e-13, max_cycles=2000, max_outer=1)
    got = psi64.cpu().numpy()
    errs = [rel(got[g], ref[g]) for g in range(gp.G)]
    print("per-group relative error vs FP64 oracle (%s):" % code, ["%.2e" % e for e in errs])
    assert max(errs) < 1e-8, errs


def test_refinement_goes_below_the_fp32_floor():
    """Plain FP32 cycles stall at the FP32 rounding floor of the residual;
    BF16 inner cycles with the FP64 outer residual reach 1e-9."""
    prob = I.checkerboard(n=64, n_polar=8, n_azim=16, blocks=4, seed=2, c=0.9)
    gp32 = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    psi = gp32.zeros()
    plain = gp32.solve(psi, rtol=1e-9, max_cycles=300)
    gpb = btmg.Problem(prob, dtype=btmg.BF16, pg=0)
    psi64 = torch.zeros(gpb.shape, dtype=torch.float64, device="cuda")
    refined = gpb.solve_refined(psi64, rtol=1e-9, max_outer=120, inner_cycles=4)
    print("plain FP32 final residual %.2e after %d cycles; refined BF16 %.2e after %d inner cycles"
          % (plain["rel_resid"], plain["cycles"], refined["rel_resid"], refined["cycles"]))
    assert refined["status"] == btmg.OK and refined["rel_resid"] <= 1e-9
    assert plain["rel_resid"] > refined["rel_resid"]


def test_refinement_rejects_pg():
    prob = I.uniform(8, 8, 4, 8)
    gp = btmg.Problem(prob, dtype=btmg.BF16, pg=1)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(btmg.BtmgError) as e:
        gp.solve_refined(psi64)
    assert e.value.code == btmg.ERR_UNSUPPORTED
