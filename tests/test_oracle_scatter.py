"""Pins of the oracle's scattering smoother variant (CPU only).

The method as published has no scattering in the upwind correction sweeps;
the variant (scat_levels = 1: levels of the coarsest angular resolution,
2: every level) solves each node's directions together with their in-node
isotropic scattering sigma_s phi / (4 pi), neighbours lagged.  Pinned
against what the definition fixes, never against the oracle's own closed
form:

S1  coarse scattering ratio = mean of the present children's sigma_s/sigma_t
S2  a sweep satisfies the node equations it is defined by
S3  many sweeps converge to a dense direct solve of (A_up - S) delta = s
S4  sigma_s = 0 gives the plain upwind Jacobi sweep
S5  scat_levels = 1 touches only the levels with N_r = N_c = 1
S6  the variant solves the same fine equations (same solution), in fewer
    cycles, and in far fewer where scattering dominates
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_09991_gb300 import inputs as I

PI = np.pi


def _pool_mean(c):
    """Mean over the present children of 2x2 blocks (ceil(n/2) each way)."""
    ny, nx = c.shape
    fy, fx = (2 if ny > 1 else 1), (2 if nx > 1 else 1)
    Y, X = -(-ny // fy), -(-nx // fx)
    acc, cnt = np.zeros((Y, X)), np.zeros((Y, X))
    for b in range(fy):
        for a in range(fx):
            sub = c[b::fy, a::fx]
            acc[:sub.shape[0], :sub.shape[1]] += sub
            cnt[:sub.shape[0], :sub.shape[1]] += 1
    return acc / cnt


def _diag(lv):
    return (np.abs(lv["mu"])[:, None, None] / lv["dx"] + np.abs(lv["nu"])[:, None, None] / lv["dy"]
            + lv["sigt"][0][None])


def test_s1_coarse_scattering_ratio():
    prob = I.checkerboard(n=13, ny=9, n_polar=8, n_azim=8, blocks=3, seed=4, c=0.8)
    # vary the ratio per region so the mean is not trivially constant
    prob["sigma_s"] = prob["sigma_s"] * np.linspace(0.5, 1.2, len(prob["sigma_t"]))[:, None, None]
    op = O.OracleProblem(prob, pg=0, scat_levels=2)
    st = prob["sigma_t"][prob["region"], 0]
    ss = prob["sigma_s"][prob["region"], 0, 0]
    c = ss / st
    for l, lv in enumerate(op.levels):
        if l > 0:
            c = _pool_mean(c)
        np.testing.assert_allclose(lv["cratio"][0], c, rtol=1e-14)


def _small_level_problem(c=0.9, scat_levels=2, bc=(0, 0, 0, 0)):
    prob = I.checkerboard(n=8, ny=6, n_polar=8, n_azim=8, blocks=2, seed=9, c=c, length=3.0)
    prob["bc"] = bc
    return prob, O.OracleProblem(prob, pg=0, scat_levels=scat_levels)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 0, 0, 1)])
def test_s2_sweep_solves_node_equations(bc):
    prob, op = _small_level_problem(bc=bc)
    rng = np.random.default_rng(2)
    for l in (0, 1, op.L - 1):
        lv = op.levels[l]
        shp = (lv["nd"], lv["ny"], lv["nx"])
        s, old = rng.standard_normal(shp), rng.standard_normal(shp)
        new = op.jacobi_upwind(l, 0, s, old, 1)
        D = _diag(lv)
        kappa = lv["cratio"][0] * lv["sigt"][0] / (4 * PI)
        lhs = D * new - kappa[None] * np.einsum("n,nyx->yx", lv["p"], new)[None]
        rhs = s + D * old - op.upwind_apply(l, old)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())


def test_s3_fixed_point_equals_dense_solve():
    prob, op = _small_level_problem(c=0.95)
    l = 1
    lv = op.levels[l]
    shp = (lv["nd"], lv["ny"], lv["nx"])
    n = int(np.prod(shp))
    # dense A_up - S, column by column: A_up from the upwind operator, S from
    # the definition sigma_s / (4 pi) sum_m p_m delta_m at the same node
    kappa = lv["cratio"][0] * lv["sigt"][0] / (4 * PI)
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        E = e.reshape(shp)
        M[:, j] = (op.upwind_apply(l, E) - kappa[None] * np.einsum("n,nyx->yx", lv["p"], E)[None]).ravel()
    s = np.random.default_rng(5).standard_normal(shp)
    direct = np.linalg.solve(M, s.ravel()).reshape(shp)
    it = op.jacobi_upwind(l, 0, s, np.zeros(shp), 400)
    np.testing.assert_allclose(it, direct, rtol=1e-9, atol=1e-11 * np.abs(direct).max())


def test_s4_no_scattering_is_plain_jacobi():
    prob = I.checkerboard(n=8, ny=6, n_polar=8, n_azim=8, blocks=2, seed=9, c=0.0)
    a = O.OracleProblem(prob, pg=0, scat_levels=2)
    b = O.OracleProblem(prob, pg=0, scat_levels=0)
    rng = np.random.default_rng(1)
    for l in range(a.L):
        lv = a.levels[l]
        shp = (lv["nd"], lv["ny"], lv["nx"])
        s, d = rng.standard_normal(shp), rng.standard_normal(shp)
        np.testing.assert_allclose(a.jacobi_upwind(l, 0, s, d, 3), b.jacobi_upwind(l, 0, s, d, 3),
                                   rtol=1e-14, atol=1e-14)


def test_s5_coarsest_angle_only():
    prob = I.checkerboard(n=8, ny=6, n_polar=8, n_azim=16, blocks=2, seed=9, c=0.9)
    one = O.OracleProblem(prob, pg=0, scat_levels=1)
    two = O.OracleProblem(prob, pg=0, scat_levels=2)
    off = O.OracleProblem(prob, pg=0, scat_levels=0)
    rng = np.random.default_rng(8)
    seen = set()
    for l in range(one.L):
        lv = one.levels[l]
        shp = (lv["nd"], lv["ny"], lv["nx"])
        s, d = rng.standard_normal(shp), rng.standard_normal(shp)
        coarsest = lv["nr"] == 1 and lv["nc"] == 1
        ref = (two if coarsest else off).jacobi_upwind(l, 0, s, d, 2)
        np.testing.assert_array_equal(one.jacobi_upwind(l, 0, s, d, 2), ref)
        seen.add(coarsest)
    assert seen == {True, False}


def test_s6_same_solution_fewer_cycles():
    prob = I.checkerboard(n=24, n_polar=8, n_azim=8, blocks=4, seed=3, c=0.9, length=5.0)
    plain = O.OracleProblem(prob, pg=0)
    var = O.OracleProblem(prob, pg=0, scat_levels=2)
    p0, n0, r0, _ = plain.solve(rtol=1e-11, max_cycles=2000)
    p1, n1, r1, _ = var.solve(rtol=1e-11, max_cycles=2000)
    assert r0 < 1e-11 and r1 < 1e-11
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-9 * np.abs(p0).max())
    assert n1 < n0
    # scattering-dominated and optically thick: the plain cycle stalls on
    # the slow isotropic mode that the variant's sweeps carry
    thick = I.checkerboard(n=32, n_polar=8, n_azim=8, blocks=4, seed=3, c=0.99, length=30.0)
    _, na, ra, _ = O.OracleProblem(thick, pg=0).solve(rtol=1e-6, max_cycles=200)
    _, nb, rb, _ = O.OracleProblem(thick, pg=0, scat_levels=2).solve(rtol=1e-6, max_cycles=200)
    print("c = 0.99, side 30: plain %d cycles (%.1e), variant %d cycles (%.1e)" % (na, ra, nb, rb))
    assert rb < 1e-6 and nb <= 40
    assert ra > 1e-6
