"""Batched solves (GPU): many independent problems of uneven grid and angular
sizes advanced together by one graph launch per cycle.

- Every problem of a batch ends bit-for-bit where the same number of plain
  btmg_mg_cycle calls on its own leaves it (same kernels, same chunking).
- A converged FP64 batch member matches the FP64 oracle's converged solve.
- The autotuner picks a valid chunk count and does not change the solution
  beyond FP32 rounding.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu


def _rel_resid(gp, prob, psi):
    """||b - A psi||_W / ||q||_W with W = p_n dx dy (dx dy cancels)."""
    r = gp.apply_operator(psi).double()
    p = torch.tensor(gp.levels[0]["p"], dtype=torch.float64, device="cuda")
    num = float((p[None, :, None, None] * r * r).sum())
    q = np.asarray(prob["source"])[np.asarray(prob["region"])]  # [ny][nx][G]
    den = 4.0 * np.pi * float((q * q).sum())
    return (num / den) ** 0.5


def _mixed(seed=4, count=5):
    """Voronoi problems of uneven sizes and direction grids (the batched
    workload family at sizes the test finishes in seconds)."""
    rng = np.random.default_rng(seed)
    grids = ((4, 8), (8, 8), (8, 16), (16, 16))
    out = []
    for i in range(count):
        n = int(rng.choice([24, 40, 48, 56, 72]))
        g = grids[int(rng.integers(len(grids)))]
        out.append(I.voronoi(n, g[0], g[1], seed * 1000003 + i))
    return out


@pytest.mark.parametrize("pg", [0, 1])
def test_batch_matches_individual_cycles_bitwise(pg):
    probs = _mixed()
    b = btmg.Batch(probs, dtype=btmg.F32, pg=pg)
    psis = b.zeros()
    max_cycles = 60 if pg else 400
    rc, infos = b.solve(psis, rtol=1e-5, max_cycles=max_cycles, check_every=1)
    for i, (prob, info) in enumerate(zip(probs, infos)):
        c, _, _ = b.chunks(i)
        gp = btmg.Problem(prob, dtype=btmg.F32, pg=pg, chunks=c)
        psi = gp.zeros()
        for _ in range(info["cycles"]):
            gp.mg_cycle(psi, want_residual=False)
        torch.cuda.synchronize()
        assert torch.equal(psi, psis[i]), (i, info)
        if pg == 0:
            assert info["status"] == btmg.OK and info["rel_resid"] <= 1e-5, info
        # the reported residual is the residual of the returned psi
        r = _rel_resid(gp, prob, psis[i])
        assert abs(info["rel_resid"] - r) <= 1e-5 * max(r, 1e-30), (info, r)


def test_persistent_coarse_launch_is_used_and_matches_single_cycles_bf16():
    """Batches of one-group FP32-compute problems run their coarse
    corrections in the persistent launch; with BF16 storage every member
    still equals its own cycles bit for bit; autotuning picks a tile width
    of 16 or 32 and 1, 2 or 4 CTAs per SM."""
    probs = _mixed(seed=6, count=6)
    b = btmg.Batch(probs, dtype=btmg.BF16, pg=0, autotune=True)
    psis = b.zeros()
    rc, infos = b.solve(psis, rtol=0.0, max_cycles=5, check_every=5)
    persistent, tile, ctas, ms = b.coarse()
    assert persistent and tile in (16, 32) and ctas in (1, 2, 4) and ms > 0, (persistent, tile, ctas, ms)
    for i, (prob, info) in enumerate(zip(probs, infos)):
        gp = btmg.Problem(prob, dtype=btmg.BF16, pg=0, chunks=b.chunks(i)[0])
        psi = gp.zeros()
        for _ in range(info["cycles"]):
            gp.mg_cycle(psi, want_residual=False)
        torch.cuda.synchronize()
        assert torch.equal(psi, psis[i]), (i, info)
    # FP64 and multigroup batches keep a whole cycle per graph branch
    assert not btmg.Batch(probs[:2], dtype=btmg.F64, pg=0).coarse()[0]
    assert not btmg.Batch([I.multigroup(n=24, n_polar=4, n_azim=8, G=2, blocks=3, seed=7)],
                          dtype=btmg.F32, pg=0).coarse()[0]


def test_batch_f64_member_matches_oracle_solve():
    probs = [I.voronoi(24, 4, 8, 77), I.voronoi(40, 8, 8, 78), I.two_region(nx=20, ny=28)]
    b = btmg.Batch(probs, dtype=btmg.F64, pg=0)
    psis = b.zeros()
    rc, infos = b.solve(psis, rtol=1e-11, max_cycles=3000, check_every=5)
    assert rc == btmg.OK, infos
    for k in (0, 2):
        op = O.OracleProblem(probs[k], pg=0)
        ref, n, r, _ = op.solve(rtol=1e-11, max_cycles=3000)
        got = psis[k].cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print("batch member %d vs oracle: %.2e (oracle %d cycles, batch %d)" % (k, err, n, infos[k]["cycles"]))
        assert err < 1e-9


def test_autotuned_chunks_are_valid_and_keep_the_solution():
    probs = _mixed(seed=9, count=3)
    ref = btmg.Batch(probs, dtype=btmg.F32, pg=0)
    tuned = btmg.Batch(probs, dtype=btmg.F32, pg=0, autotune=True)
    pr, pt = ref.zeros(), tuned.zeros()
    ref.solve(pr, rtol=1e-5, max_cycles=400)
    tuned.solve(pt, rtol=1e-5, max_cycles=400)
    for i, p in enumerate(tuned.problems):
        c, a, ms = tuned.chunks(i)
        assert 1 <= c <= 64 and p.nd % c == 0 and 4 * c >= a and c <= 4 * a and ms > 0, (c, a, ms)
        diff = float(torch.linalg.norm(pt[i] - pr[i]) / torch.linalg.norm(pr[i]))
        assert diff < 1e-4, (i, diff)


def test_batch_argument_errors():
    prob = I.voronoi(24, 4, 8, 5)
    with pytest.raises(btmg.BtmgError) as e:
        btmg.Problem(prob, dtype=btmg.F32, pg=0, chunks=7)  # 32 directions: 7 does not divide
    assert e.value.code == btmg.ERR_INVALID_ARG
    b = btmg.Batch([prob], dtype=btmg.F32, pg=0)
    with pytest.raises(ValueError):
        b.solve([])
