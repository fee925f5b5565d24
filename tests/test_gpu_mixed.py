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


def test_full_size_mixed_precision_sampled_planes():
    """The mixed-precision workload at full size: 512^2 nodes, 32 x 32
    directions, 4 downscatter groups (1.07 G unknowns), psi in BF16 with
    FP32 accumulation, FP64 refinement to 1e-6.  The FP64 oracle, which
    cannot solve this size in a test, evaluates the residual of the returned
    FP64 solution on 12 sampled (group, direction) planes: it must equal the
    GPU's FP64 residual there, and be small against the planes' source."""
    prob = I.multigroup(n=512, n_polar=32, n_azim=32, G=4, seed=3)
    gp = btmg.Problem(prob, dtype=btmg.BF16, pg=0)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    out = gp.solve_refined(psi64, rtol=1e-6, max_outer=100, inner_cycles=32)
    print("full-size BF16 refined solve: status %d, rel %.2e, %d inner cycles"
          % (out["status"], out["rel_resid"], out["cycles"]))
    assert out["status"] == btmg.OK and out["rel_resid"] <= 1e-6, out
    del gp
    g64 = btmg.Problem(prob, dtype=btmg.F64, pg=0)
    r_gpu = g64.apply_operator(psi64)
    rng = np.random.default_rng(3)
    planes = [(int(g), int(n)) for g, n in zip(rng.integers(0, 4, 12), rng.choice(g64.nd, 12, replace=False))]
    got = np.stack([r_gpu[g, n].cpu().numpy() for g, n in planes])
    del r_gpu, g64
    torch.cuda.empty_cache()
    op = O.OracleProblem(prob, pg=0)
    ref = op.apply_planes(psi64.cpu().numpy(), planes)
    # the residual is a difference of terms of the size of the source, so
    # the two FP64 evaluations (different summation orders) agree to a few
    # ulps of those terms, not of the much smaller residual itself
    q0 = np.linalg.norm(np.asarray(prob["source"])[np.asarray(prob["region"])][..., 0])
    for (g, n), a, b in zip(planes, got, ref):
        print("plane (%d, %d): |r|/|q| = %.2e, |r_gpu - r_oracle|/|q| = %.2e"
              % (g, n, np.linalg.norm(b) / q0, np.linalg.norm(a - b) / q0))
        assert np.linalg.norm(a - b) <= 1e-11 * q0, (g, n, np.linalg.norm(a - b) / q0)
    # one plane carries at most the whole weighted residual: with weight
    # p_n ~ 4 pi / 1024 and ||r||_W <= 1e-6 ||q||_W, a plane's residual stays
    # below ~3e-5 ||q||; the external source of group 0 sets the scale
    for (g, n), r in zip(planes, ref):
        assert np.linalg.norm(r) <= 1e-4 * q0, (g, n, np.linalg.norm(r) / q0)
    # particle balance of the refined solution on the GPU (FP64, per group):
    # production = removal + leakage to the residual level
    g64 = btmg.Problem(prob, dtype=btmg.F64, pg=0)
    bal = g64.particle_balance(psi64)
    print("particle balance per group (production, removal, leakage, imbalance):\n", bal)
    assert np.all(np.abs(bal[:, 3]) < 1e-5)
