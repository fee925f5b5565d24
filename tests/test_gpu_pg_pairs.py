"""GPU parity of the FP32 PG operator on direction pairs (the packed FP32x2
kernel), of FP32 PG cycles at the full 256^2 x 512 workload, and of converged
FP32 solves at the workload's angular resolution.

The paired kernel runs whenever a chunk holds an even number of directions
and rows are 16-byte multiples; a chunk count that leaves an odd number of
directions per chunk routes the same problem to the single-direction kernel,
so both are compared with the FP64 oracle and with each other on the same
input.
"""
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


def host(t):
    return t.double().cpu().numpy()


def odd_chunks(nd):
    """A chunk count (at most 64) that leaves an odd number of directions per chunk."""
    return max(c for c in range(1, 65) if nd % c == 0 and (nd // c) % 2 == 1)


PAIR_CASES = [
    # partial tiles in both axes, vacuum
    ("checker_68x37_72dirs", lambda: I.checkerboard(n=68, ny=37, n_polar=6, n_azim=12, blocks=4, seed=31)),
    # reflective on three sides, one direction per face pair straddling faces
    ("reflective_44x20_8dirs", lambda: I.checkerboard(n=44, ny=20, n_polar=2, n_azim=4, blocks=2, seed=32,
                                                      bc=(1, 1, 0, 1))),
    ("two_region_32", lambda: I.two_region()),
]


@pytest.mark.parametrize("name,mk", PAIR_CASES)
def test_paired_kernel_residual_and_jacobi(name, mk):
    prob = mk()
    op = O.OracleProblem(prob)
    nd = prob["n_polar"] * prob["n_azim"]
    paired = btmg.Problem(prob, dtype=btmg.F32)
    single = btmg.Problem(prob, dtype=btmg.F32, chunks=odd_chunks(nd))
    psi0 = I.random_field(paired.shape, seed=33).astype(np.float32)
    ref = op.apply(psi0.astype(np.float64))
    r_pair = host(paired.apply_operator(torch.tensor(psi0, device="cuda")))
    r_single = host(single.apply_operator(torch.tensor(psi0, device="cuda")))
    assert rel(r_pair, ref) < 1e-6
    assert rel(r_single, ref) < 1e-6
    assert rel(r_pair, r_single) < 1e-6
    # one PG Jacobi sweep (beta = 3) from the same psi
    jref = op.pg_jacobi(psi0.astype(np.float64), 1)
    for gp in (paired, single):
        psi = torch.tensor(psi0, device="cuda")
        gp.smooth_pg(psi, sweeps=1)
        assert rel(host(psi), jref) < 1e-6


def test_fp32_pg_cycles_full_size_sampled_planes():
    """256^2 nodes x 512 directions, PG on, FP32, the benchmark's launch
    configuration: psi after one and after two cycles from psi = 0 against
    the FP64 oracle's cycles on 12 sampled (group, direction) planes.  The
    nonlinear PG cycle amplifies a perturbation of its input about 20x per
    cycle (FP64 oracle), so the second cycle's bound is 20x the first's."""
    prob = I.checkerboard(n=256, n_polar=16, n_azim=32, blocks=8, seed=2)
    gp = btmg.Problem(prob, dtype=btmg.F32)
    op = O.OracleProblem(prob)
    rng = np.random.default_rng(1)
    planes = [int(n) for n in rng.choice(gp.nd, 12, replace=False)]
    psi = gp.zeros()
    ref = op.zeros()
    for k, tol in enumerate((1e-5, 2e-4)):
        gp.mg_cycle(psi)
        ref, _, _ = op.mg_cycle(ref)
        got = np.stack([host(psi[0, n]) for n in planes])
        want = np.stack([ref[0, n] for n in planes])
        assert rel(got, want) < tol, (k, rel(got, want))


def test_converged_fp32_solve_at_16x32_directions():
    """128^2 nodes, 16 x 32 directions (the workload's angular resolution),
    checkerboard, c = 0.9, upwind fine scheme: plain FP32 cycles to the FP32
    floor and FP64-refined FP32 cycles, against the oracle's converged FP64
    solve (relative residual 1e-11): within 1e-5 and 1e-8."""
    prob = I.checkerboard(n=128, n_polar=16, n_azim=32, blocks=4, seed=2, c=0.9)
    op = O.OracleProblem(prob, pg=0)
    ref, n, rr, _ = op.solve(rtol=1e-11, max_cycles=400)
    assert rr < 1e-11
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    psi = gp.zeros()
    out = gp.solve(psi, rtol=1e-7, max_cycles=300)
    assert out["status"] in (btmg.OK, btmg.ERR_NOT_CONVERGED)
    assert rel(host(psi), ref) < 1e-5, out["rel_resid"]
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    r = gp.solve_refined(psi64, rtol=1e-10, max_outer=60, inner_cycles=16)
    assert r["rel_resid"] <= 1e-10
    assert rel(host(psi64), ref) < 1e-8
