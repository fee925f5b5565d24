"""Scattering smoother (desc.scat_levels, a variant of the upwind correction
sweeps) on the GPU against the FP64 oracle: every level's node-block
sweeps element by element, cycle sequences, converged solves, and the
convergence gain in the scattering-dominated regime.

Tolerances (relative L2): FP64 sweeps 1e-13, FP64 cycles 1e-10 (rounding
order only: the scalar flux of a sweep is summed per direction chunk on the
GPU, over all directions at once in the oracle); FP32 sweeps 1e-5 (2-ulp
reciprocal of the diagonal, FP32 sums over up to 512 directions)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


CASES = [
    ("checker_72x40", lambda: I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=11, c=0.95,
                                             length=4.0)),
    ("tiny_5x3", lambda: I.checkerboard(n=5, ny=3, n_polar=4, n_azim=8, blocks=2, seed=12)),
    ("one_node", lambda: I.uniform(1, 1, 2, 4, sigma_t=1.3, c=0.4)),
    ("reflective_33x17", lambda: I.checkerboard(n=33, ny=17, n_polar=4, n_azim=8, blocks=3, seed=13,
                                                bc=(1, 0, 1, 1), c=0.99)),
]


@pytest.mark.parametrize("name,mk", CASES)
@pytest.mark.parametrize("scat", [1, 2])
@pytest.mark.parametrize("sweeps", [1, 3, 4])
def test_smoother_every_level_fp64(name, mk, scat, sweeps):
    prob = mk()
    gp = btmg.Problem(prob, dtype=btmg.F64, scat_levels=scat)
    op = O.OracleProblem(prob, scat_levels=scat)
    rng = np.random.default_rng(sweeps + 10 * scat)
    for l in range(gp.L):
        s = rng.standard_normal(gp.level_shape(l))
        d0 = rng.standard_normal(gp.level_shape(l))
        d = dev(d0, torch.float64)
        gp.smooth_upwind(d, dev(s, torch.float64), l, 0, sweeps)
        assert rel(host(d), op.jacobi_upwind(l, 0, s, d0, sweeps)) < 1e-13, l


def test_smoother_every_level_fp32():
    prob = I.checkerboard(n=96, ny=70, n_polar=16, n_azim=32, blocks=4, seed=3, c=0.98, length=10.0)
    gp = btmg.Problem(prob, dtype=btmg.F32, scat_levels=2)
    op = O.OracleProblem(prob, scat_levels=2)
    rng = np.random.default_rng(4)
    for l in range(gp.L):
        s = rng.standard_normal(gp.level_shape(l)).astype(np.float32)
        d0 = rng.standard_normal(gp.level_shape(l)).astype(np.float32)
        d = dev(d0, torch.float32)
        gp.smooth_upwind(d, dev(s, torch.float32), l, 0, 3)
        assert rel(host(d), op.jacobi_upwind(l, 0, s, d0, 3)) < 1e-5, l


@pytest.mark.parametrize("name,mk", CASES)
@pytest.mark.parametrize("pg", [1, 0])
@pytest.mark.parametrize("scat", [1, 2])
def test_mg_cycle_sequence_fp64(name, mk, pg, scat):
    prob = mk()
    gp = btmg.Problem(prob, dtype=btmg.F64, pg=pg, scat_levels=scat)
    op = O.OracleProblem(prob, pg=pg, scat_levels=scat)
    psi = gp.zeros()
    ref = op.zeros()
    for k in range(3):
        rg = gp.mg_cycle(psi)
        ref, rr, _ = op.mg_cycle(ref)
        assert abs(rg - rr) <= 1e-9 * max(rr, 1e-30), (k, rg, rr)
        assert rel(host(psi), ref) < 1e-10, k


@pytest.mark.parametrize("n,ny,bc", [(96, 72, (0, 0, 0, 0)), (100, 37, (1, 0, 0, 1)), (132, 20, (0, 1, 1, 0))])
def test_mg_cycle_sequence_fp32_four_node_kernels(n, ny, bc):
    """x sizes that are multiples of 4 take the four-nodes-per-thread FP32
    kernels (first sweep from the UpSamp, sweeps from J, final pass);
    ragged tiles and reflective sides included."""
    prob = I.checkerboard(n=n, ny=ny, n_polar=8, n_azim=16, blocks=4, seed=21, c=0.97, length=6.0, bc=bc)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, scat_levels=2)
    op = O.OracleProblem(prob, pg=0, scat_levels=2)
    psi = gp.zeros()
    ref = op.zeros()
    for k in range(3):
        gp.mg_cycle(psi)
        ref, _, _ = op.mg_cycle(ref)
        assert rel(host(psi), ref) < 1e-5, k


def test_mg_cycle_multigroup_fp64():
    prob = I.multigroup(n=24, n_polar=4, n_azim=8, G=3, blocks=3, seed=5)
    gp = btmg.Problem(prob, dtype=btmg.F64, pg=0, scat_levels=2)
    op = O.OracleProblem(prob, pg=0, scat_levels=2)
    psi = gp.zeros()
    ref = op.zeros()
    for _ in range(2):
        gp.mg_cycle(psi)
        ref, _, _ = op.mg_cycle(ref)
    assert rel(host(psi), ref) < 1e-10


def test_converged_solve_matches_oracle_and_plain_solution():
    """Scattering-dominated, 30 mean free paths of the thickest block: the
    variant's FP64 solve takes the oracle's number of cycles and lands on
    the oracle's solution, which is the solution of the unchanged fine
    equations (the plain cycle's, to its own tolerance)."""
    prob = I.checkerboard(n=40, n_polar=8, n_azim=16, blocks=4, seed=3, c=0.99, length=30.0)
    gp = btmg.Problem(prob, dtype=btmg.F64, pg=0, scat_levels=2)
    op = O.OracleProblem(prob, pg=0, scat_levels=2)
    psi = gp.zeros()
    out = gp.solve(psi, rtol=1e-10, max_cycles=400)
    ref, n, rr, _ = op.solve(rtol=1e-10, max_cycles=400)
    assert out["status"] == btmg.OK and rr < 1e-10
    assert abs(out["cycles"] - n) <= 1, (out["cycles"], n)
    assert rel(host(psi), ref) < 1e-9
    plain = btmg.Problem(prob, dtype=btmg.F64, pg=0)
    p0 = plain.zeros()
    o0 = plain.solve(p0, rtol=1e-10, max_cycles=20000, check_every=50)
    print("c = 0.99, side 30, 40^2 x 128: variant %d cycles, plain %d cycles" % (out["cycles"], o0["cycles"]))
    assert o0["status"] == btmg.OK
    assert rel(host(psi), host(p0)) < 1e-8
    assert out["cycles"] * 10 < o0["cycles"]


def test_fp32_thick_gain_and_refined_bf16():
    prob = I.checkerboard(n=128, n_polar=16, n_azim=32, blocks=8, seed=5, c=0.99, length=30.0)
    res = {}
    # FP32 rounds this problem's residual to a floor near 1.3e-5: solve to 3e-5
    for scat in (0, 2):
        gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, scat_levels=scat)
        psi = gp.zeros()
        res[scat] = gp.solve(psi, rtol=3e-5, max_cycles=400, history=False)
    print("FP32 to 3e-5: plain %s, variant %s" % (res[0], res[2]))
    assert res[2]["status"] == btmg.OK and res[2]["cycles"] <= 40
    assert res[0]["status"] != btmg.OK or res[0]["cycles"] > 5 * res[2]["cycles"]
    gb = btmg.Problem(prob, dtype=btmg.BF16, pg=0, scat_levels=2)
    psi64 = torch.zeros(gb.shape, dtype=torch.float64, device="cuda")
    out = gb.solve_refined(psi64, rtol=1e-8, max_outer=60, inner_cycles=8)
    print("BF16 refined to 1e-8 with the variant:", out)
    assert out["status"] == btmg.OK and out["rel_resid"] <= 1e-8


def test_batch_members_equal_single_cycles():
    probs = [I.checkerboard(n=n, n_polar=8, n_azim=16, blocks=4, seed=20 + n, c=0.98, length=10.0)
             for n in (24, 40, 57)]
    b = btmg.Batch(probs, dtype=btmg.F32, pg=0, scat_levels=2)
    psis = [p.zeros() for p in b.problems]
    _, infos = b.solve(psis, rtol=1e-5, max_cycles=6, check_every=1)
    for prob, psi, info in zip(probs, psis, infos):
        gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, scat_levels=2)
        q = gp.zeros()
        for _ in range(info["cycles"]):
            gp.mg_cycle(q)
        assert torch.equal(psi, q)


def test_plain_multigrid_arbitrates_the_smoother():
    """Thin unit square at 512^2 x 1024 directions, c = 0.9: the smoother's
    cycle grows the residual in mid-solve (a transient the published cycle
    also shows, weaker); the solve drops it when the residual passes twice
    (unrefined) or 1.5 times (refined) its best and still converges."""
    prob = I.checkerboard(n=512, n_polar=32, n_azim=32, blocks=8, seed=5000, c=0.9)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, scat_levels=2)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    out = gp.solve_refined(psi64, rtol=1e-6, max_outer=40, inner_cycles=32)
    print("refined:", out["status"], out["cycles"], out["rel_resid"], gp.scatter_fallbacks())
    assert out["status"] == btmg.OK and gp.scatter_fallbacks() == 1
    psi = gp.zeros()
    out = gp.solve(psi, rtol=1e-3, max_cycles=1500, check_every=5, history=False)
    print("plain solve:", out["status"], out["cycles"], out["rel_resid"], gp.scatter_fallbacks())
    assert out["status"] == btmg.OK and gp.scatter_fallbacks() == 2
    # the next solve starts with the smoother again: a cycle of it matches
    # the oracle's smoother cycle on a small problem of the same family
    small = I.checkerboard(n=24, n_polar=8, n_azim=8, blocks=4, seed=5, c=0.9)
    g2 = btmg.Problem(small, dtype=btmg.F64, pg=0, scat_levels=2)
    q = g2.zeros()
    g2.solve(q, rtol=1e-30, max_cycles=3)
    op = O.OracleProblem(small, pg=0, scat_levels=2)
    ref = op.zeros()
    for _ in range(3):
        ref, _, _ = op.mg_cycle(ref)
    assert g2.scatter_fallbacks() == 0 and rel(host(q), ref) < 1e-10


def test_invalid_scat_levels():
    prob = I.uniform(8, 8, 4, 8, sigma_t=1.0, c=0.5)
    with pytest.raises(btmg.BtmgError) as e:
        btmg.Problem(prob, dtype=btmg.F32, scat_levels=3)
    assert e.value.code == btmg.ERR_INVALID_ARG
    bad = dict(prob)
    bad["sigma_s"] = prob["sigma_s"] * 3.0  # sigma_s > sigma_t
    with pytest.raises(btmg.BtmgError) as e:
        btmg.Problem(bad, dtype=btmg.F32, scat_levels=2)
    assert e.value.code == btmg.ERR_INVALID_ARG
    btmg.Problem(bad, dtype=btmg.F32, scat_levels=0)  # the plain cycle accepts it
