"""Pins of the FP64 CPU oracle against what the paper and the mathematics
fix (never against the oracle itself).  CPU only.

P1  filters equal the paper's printed Appendix tables (A.1, A.2, A.3)
P2  filters are consistent on polynomials (signs and orientation)
P3  quadrature: closed-form octant area, symmetry, self-convergence (Sec. 2.2)
P4  infinite medium: psi = s / (sigma_t - sigma_s) is the fixed point; with
    three groups (down- and upscatter) the 3 x 3 system's solution
P5  upwind mode converges to an independent transport sweep
P6  frozen-k linear system: MG fixed point equals a dense direct solve
P7  particle balance of the upwind discretisation
P8  manufactured solution: ConvFEM + PG operator is 4th-order consistent
P9  D4 symmetry of the cycle on a symmetric problem
P10 restriction / UpSamp adjointness; coarsest 1x1 Jacobi gives s/d
P11 PG coefficients k_x on a quintic with closed-form Psi_x and R_x
"""
import numpy as np
import pytest

import oracle as O
from golden.load import load_blocks
from paper_2301_09991_gb300 import inputs as I

PI = np.pi


# ---------------------------------------------------------------- P1 -----
def _close_3sf(printed, exact):
    """Printed 3-significant-figure values: within 0.5 % (and exact zeros)."""
    zero = printed == 0
    assert np.all(np.abs(exact[zero]) < 1e-12)
    rel = np.abs(printed[~zero] - exact[~zero]) / np.abs(exact[~zero])
    assert rel.max() < 5e-3, rel.max()


def test_p1_quadratic_filters_match_appendix_a2():
    g = load_blocks("quadratic_filters.txt")
    f = O.filters_2d(2, 1.0, 1.0)
    # w_x: columns are x offsets, rows y offsets (-2 top); w_y likewise.
    for k in ("wx", "wy", "wdxx", "wdyy", "wm"):
        _close_3sf(g[k], f[k])


def test_p1_linear_filters_match_appendix_a1():
    g = load_blocks("linear_filters.txt")
    f = O.filters_2d(1, 1.0, 1.0)
    _close_3sf(g["wdxx"], f["wdxx"])
    _close_3sf(g["wdyy"], f["wdyy"])
    _close_3sf(g["wm"], f["wm"])
    # printed w_x is twice the FEM value (reading: use the derived filter)
    _close_3sf(g["wx"], 2.0 * f["wx"])
    # printed w_y has +y on the top row
    _close_3sf(g["wy"], 2.0 * f["wy"][::-1, :])


def test_p1_cubic_wx_matches_appendix_a3():
    g = load_blocks("cubic_wx.txt")
    f = O.filters_2d(3, 1.0, 1.0)
    _close_3sf(g["wx"], f["wx"])


def test_p1_quadratic_stencils_rational():
    m1, d1, s1, ml = O.convfem_1d(2)
    np.testing.assert_allclose(m1, [-1 / 30, 2 / 15, 4 / 5, 2 / 15, -1 / 30], atol=1e-14)
    np.testing.assert_allclose(d1, [1 / 12, -2 / 3, 0, 2 / 3, -1 / 12], atol=1e-14)
    np.testing.assert_allclose(s1, [1 / 12, -4 / 3, 5 / 2, -4 / 3, 1 / 12], atol=1e-13)
    assert abs(ml - 1.0) < 1e-13  # lumped mass per node = h


# ---------------------------------------------------------------- P2 -----
@pytest.mark.parametrize("order", [1, 2, 3])
def test_p2_filters_on_polynomials(order):
    h = 0.37
    f = O.filters_2d(order, h, h)
    l = order
    off = np.arange(-l, l + 1) * h
    X, Y = np.meshgrid(off + 0.3, off - 0.2)  # values around (0.3, -0.2)
    corr = lambda w, a: float(np.sum(w * a))
    assert abs(corr(f["wx"], X) - 1.0) < 1e-12  # d/dx x = 1
    assert abs(corr(f["wy"], Y) - 1.0) < 1e-12
    assert abs(corr(f["wx"], Y)) < 1e-12
    assert abs(corr(f["wdxx"], X ** 2 / 2) + 1.0) < 1e-11  # -d2/dx2 (x^2/2) = -1
    assert abs(corr(f["wdyy"], Y ** 2 / 2) + 1.0) < 1e-11
    assert abs(corr(f["wm"], np.ones_like(X)) - 1.0) < 1e-13
    if order >= 2:  # 4th-order consistency: exact on cubics, w_m - I kills cubics
        assert abs(corr(f["wx"], X ** 3) - 3 * 0.3 ** 2) < 1e-11
        assert abs(corr(f["wm"], X ** 3) - 0.3 ** 3) < 1e-12


# ---------------------------------------------------------------- P3 -----
def test_p3_octant_area_closed_form():
    # each octahedron face projects onto one octant of the sphere: area pi/2
    mu, nu, xi, p = O.quadrature(4, 2, ngauss=16, normalise=False)
    for f in range(8):
        assert abs(p[f * 8:(f + 1) * 8].sum() - PI / 2) < 1e-13


def test_p3_quadrature_sums_and_symmetry():
    for nr, nc in ((4, 2), (8, 8), (16, 8)):
        mu, nu, xi, p = O.quadrature(nr, nc)
        nd = 8 * nr * nc
        assert abs(p.sum() - 4 * PI) < 1e-12
        assert abs(np.dot(p, mu)) < 1e-12 and abs(np.dot(p, nu)) < 1e-12
        assert np.all(np.abs(mu) ** 2 + np.abs(nu) ** 2 + xi ** 2 <= 1 + 1e-12)
        q = nr * nc
        for f in range(8):
            sx = -1 if f & 1 else 1
            sy = -1 if f & 2 else 1
            sl = slice(f * q, (f + 1) * q)
            assert np.all(np.sign(mu[sl]) == sx) and np.all(np.sign(nu[sl]) == sy)
            # mu <-> nu under i -> nc-1-i (the a <-> b swap of the face map)
            m = mu[sl].reshape(nr, nc)
            n_ = nu[sl].reshape(nr, nc)
            np.testing.assert_allclose(np.abs(m), np.abs(n_[:, ::-1]), atol=1e-14)
            np.testing.assert_allclose(p[sl], p[:q], atol=1e-14)  # all faces alike


def test_p3_gauss_self_convergence_and_moment():
    a = O.quadrature(8, 8, ngauss=16)
    b = O.quadrature(8, 8, ngauss=32)
    for u, v in zip(a, b):
        assert np.max(np.abs(u - v)) < 1e-12
    errs = []
    for nr, nc in ((2, 1), (4, 2), (8, 4), (16, 8)):
        mu, nu, xi, p = O.quadrature(nr, nc)
        errs.append(abs(np.dot(p, mu ** 2) - 4 * PI / 3))
    assert errs[-1] < errs[0] and errs[-1] < 0.05


def test_p3_gauss_legendre_matches_numpy():
    for n in (1, 2, 5, 16):
        x, w = O.gauss01(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(np.sort(x), np.sort((xr + 1) / 2), atol=1e-14)
        np.testing.assert_allclose(np.sort(w), np.sort(wr / 2), atol=1e-14)


def test_p3_angular_coarsening_preserves_weight():
    op = O.OracleProblem(I.uniform(8, 8, 16, 32))
    for lv in op.levels:
        assert abs(lv["p"].sum() - 4 * PI) < 1e-12
        assert abs(np.dot(lv["p"], lv["mu"])) < 1e-12


# ---------------------------------------------------------------- P4 -----
@pytest.mark.parametrize("pg", [1, 0])
def test_p4_infinite_medium_closed_form(pg):
    st, c, s = 2.0, 0.6, 1.5
    # PG mode on a power-of-two grid keeps every iterate uniform; the odd
    # grid (missing coarse children) is exercised in upwind mode.
    nx, ny = (16, 8) if pg else (12, 10)
    p = I.uniform(nx, ny, 8, 8, sigma_t=st, c=c, s=s, bc=(1, 1, 1, 1))
    op = O.OracleProblem(p, pg=pg)
    exact = np.full(op.shape, s / (st - c * st))
    r = op.apply(exact)
    assert np.max(np.abs(r)) < 1e-12
    psi, n, rel, _ = op.solve(rtol=1e-13, max_cycles=200)
    assert rel < 1e-12
    np.testing.assert_allclose(psi, exact, rtol=1e-11)


@pytest.mark.parametrize("pg", [1, 0])
def test_p4_multigroup_infinite_medium_closed_form(pg):
    """Three groups with down- and upscatter ([to][from] matrix), reflective
    on every side, uniform: the flux is isotropic and constant, and per
    steradian it solves (diag(sigma_t) - Sigma_s) psi = s, a 3 x 3 system
    solved here by numpy (R3, R18)."""
    st = np.array([[1.0, 2.0, 1.5]])
    ss = np.array([[[0.3, 0.0, 0.2],     # to group 0 from 0, 1, 2 (upscatter from 2)
                    [0.4, 0.9, 0.0],     # to group 1
                    [0.1, 0.6, 0.8]]])   # to group 2
    src = np.array([[1.0, 0.5, 0.25]])
    nx, ny = (16, 8) if pg else (12, 10)
    prob = I._prob(nx, ny, 8, 8, np.zeros((ny, nx), np.int32), st, ss, src, bc=(1, 1, 1, 1))
    op = O.OracleProblem(prob, pg=pg)
    exact_g = np.linalg.solve(np.diag(st[0]) - ss[0], src[0])
    exact = np.broadcast_to(exact_g[:, None, None, None], op.shape).copy()
    assert np.max(np.abs(op.apply(exact))) < 1e-12
    psi, n, rel, _ = op.solve(rtol=1e-12, max_cycles=200, max_outer=40)
    assert rel < 1e-11
    np.testing.assert_allclose(psi, exact, rtol=1e-9)


# ---------------------------------------------------------------- P5 -----
def _sweep(op, prob):
    """Independent textbook transport sweep of the upwind scheme (sigma_s = 0,
    vacuum): each direction's system is triangular in sweep order."""
    lv = op.levels[0]
    nx, ny, dx, dy = lv["nx"], lv["ny"], lv["dx"], lv["dy"]
    st = prob["sigma_t"][prob["region"], 0]
    s = prob["source"][prob["region"], 0]
    out = np.zeros((lv["nd"], ny, nx))
    for n in range(lv["nd"]):
        mu, nu = lv["mu"][n], lv["nu"][n]
        xs = range(nx) if mu > 0 else range(nx - 1, -1, -1)
        ys = list(range(ny) if nu > 0 else range(ny - 1, -1, -1))
        for y in ys:
            for x in xs:
                up_x = x - 1 if mu > 0 else x + 1
                up_y = y - 1 if nu > 0 else y + 1
                px = out[n, y, up_x] if 0 <= up_x < nx else 0.0
                py = out[n, up_y, x] if 0 <= up_y < ny else 0.0
                a, b = abs(mu) / dx, abs(nu) / dy
                out[n, y, x] = (s[y, x] + a * px + b * py) / (a + b + st[y, x])
    return out


def test_p5_upwind_mg_equals_transport_sweep():
    prob = I.two_region(nx=12, ny=10, n_polar=8, n_azim=8, c=0.0)
    op = O.OracleProblem(prob, pg=0)
    psi, n, rel, _ = op.solve(rtol=1e-14, max_cycles=200)
    ref = _sweep(op, prob)
    np.testing.assert_allclose(psi[0], ref, rtol=1e-11, atol=1e-14)


# ---------------------------------------------------------------- P6 -----
def test_p6_frozen_k_fixed_point_equals_dense_solve():
    prob = I.two_region(nx=4, ny=4, n_polar=4, n_azim=8, c=0.5)
    op = O.OracleProblem(prob, pg=1)
    lv = op.levels[0]
    shape = op.shape
    # a frozen k field inside the stable band (0.25 k_max, varying by node)
    rng = np.random.default_rng(7)
    kx = 0.25 * lv["dx"] * np.abs(lv["mu"])[None, :, None, None] * rng.uniform(0.5, 1, shape)
    ky = 0.25 * lv["dy"] * np.abs(lv["nu"])[None, :, None, None] * rng.uniform(0.5, 1, shape)
    op.set_frozen_k(kx, ky)
    n = int(np.prod(shape))
    r0 = op.apply(np.zeros(shape)).ravel()          # = s
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = r0 - op.apply(e.reshape(shape)).ravel()
    direct = np.linalg.solve(M, r0)
    psi, cyc, rel, _ = op.solve(rtol=1e-14, max_cycles=400)
    assert rel < 1e-12
    np.testing.assert_allclose(psi.ravel(), direct, rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------- P7 -----
def test_p7_particle_balance_upwind():
    prob = I.checkerboard(n=16, n_polar=8, n_azim=8, blocks=4, seed=11, c=0.7)
    op = O.OracleProblem(prob, pg=0)
    psi, n, rel, _ = op.solve(rtol=1e-14, max_cycles=400)
    lv = op.levels[0]
    dx, dy = lv["dx"], lv["dy"]
    st = prob["sigma_t"][prob["region"], 0]
    ss = prob["sigma_s"][prob["region"], 0, 0]
    s = prob["source"][prob["region"], 0]
    phi = np.einsum("n,nyx->yx", lv["p"], psi[0])
    produced = 4 * PI * dx * dy * s.sum()
    absorbed = dx * dy * ((st - ss) * phi).sum()
    leak = 0.0
    for n_ in range(lv["nd"]):
        mu, nu, w = lv["mu"][n_], lv["nu"][n_], lv["p"][n_]
        edge_x = psi[0, n_, :, -1] if mu > 0 else psi[0, n_, :, 0]
        edge_y = psi[0, n_, -1, :] if nu > 0 else psi[0, n_, 0, :]
        leak += w * (abs(mu) * dy * edge_x.sum() + abs(nu) * dx * edge_y.sum())
    assert abs(produced - absorbed - leak) / produced < 1e-11


# ---------------------------------------------------------------- P8 -----
def _manufactured(op, B):
    lv = op.levels[0]
    x = I.node_centres(lv["nx"])[None, :]
    y = I.node_centres(lv["ny"])[:, None]
    mu = lv["mu"][:, None, None]
    nu = lv["nu"][:, None, None]
    amp = 1.0 + mu / 2 + nu / 3
    b, db = B
    psi = amp * b(x) * b(y)
    dpsi = amp * (mu * db(x) * b(y) + nu * b(x) * db(y))
    return psi[None], dpsi[None]


@pytest.mark.parametrize("order", [2, 3])
def test_p8_manufactured_order_of_consistency(order):
    """Quadratic and cubic ConvFEM + PG: a mistaken tap of the filters drops
    the observed order to 1-2; both orders measure about 4 here (the cubic
    filters are pinned to the printed w_x in P1)."""
    b = lambda t: np.sin(PI * t) ** 6
    db = lambda t: 6 * PI * np.sin(PI * t) ** 5 * np.cos(PI * t)
    errs = []
    for N in (16, 32, 64):
        prob = dict(I.uniform(N, N, 8, 8, sigma_t=0.0, c=0.0, s=0.0), order=order)
        op = O.OracleProblem(prob, pg=1)
        psi, dpsi = _manufactured(op, (b, db))
        r = op.apply(psi)  # = -(mu Psi_x + nu Psi_y + D)
        errs.append(np.sqrt(np.mean((r + dpsi) ** 2)))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order[-1] > 3.5, (errs, order)


# ---------------------------------------------------------------- P9 -----
def test_p9_d4_symmetry_of_cycles():
    prob = I.two_region(nx=16, ny=16, n_polar=8, n_azim=8)
    op = O.OracleProblem(prob, pg=1)
    psi = op.zeros()
    for _ in range(3):
        psi, rel, _ = op.mg_cycle(psi)
    phi = op.scalar_flux(psi)[0]
    scale = np.abs(phi).max()
    for t in (phi[:, ::-1], phi[::-1, :], phi.T):
        assert np.max(np.abs(t - phi)) < 1e-11 * scale


# ---------------------------------------------------------------- P10 ----
def test_p10_restriction_prolongation_adjoint():
    prob = I.checkerboard(n=10, n_polar=8, n_azim=16, blocks=2, seed=5, ny=7)
    op = O.OracleProblem(prob)
    rng = np.random.default_rng(3)
    for l in range(op.L - 1):
        A, B = op.levels[l], op.levels[l + 1]
        r = rng.standard_normal((A["nd"], A["ny"], A["nx"]))
        e = rng.standard_normal((B["nd"], B["ny"], B["nx"]))
        Rr = op.restrict(l, r)
        Ue = op.prolong(l, e)
        lhs = np.sum(B["p"][:, None, None] * B["dx"] * B["dy"] * Rr * e)
        rhs = np.sum(A["p"][:, None, None] * A["dx"] * A["dy"] * r * Ue)
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_p10_coarsest_jacobi_is_s_over_d():
    prob = I.uniform(8, 8, 8, 8, sigma_t=0.7)
    op = O.OracleProblem(prob)
    Lc = op.levels[-1]
    assert (Lc["nx"], Lc["ny"], Lc["nr"], Lc["nc"]) == (1, 1, 1, 1)
    s = np.arange(1.0, 9.0).reshape(8, 1, 1)
    d = op.jacobi_upwind(op.L - 1, 0, s, np.zeros_like(s), 3)
    diag = np.abs(Lc["mu"]) / Lc["dx"] + np.abs(Lc["nu"]) / Lc["dy"] + Lc["sigt"][0, 0, 0]
    np.testing.assert_allclose(d[:, 0, 0], s[:, 0, 0] / diag, rtol=1e-14)


# ---------------------------------------------------------------- P11 ----
@pytest.mark.parametrize("h", [0.05, 0.2, 0.6])
def test_p11_pg_coefficient_branches_on_quintic(h):
    """psi = (x - x0)^5 (any y): the 4th-order d1 gives Psi_x = 5 X^4 - 4 h^4
    exactly, the ConvFEM mass (moments 1,0,0,0,-0.8) gives
    (w_m - I) Psi_x = -4 h^4, so R_x = -12 mu h^4 and k_x follows (Eq. ano-k)."""
    N = 13
    prob = I.uniform(N, N, 4, 4, sigma_t=0.0, c=0.0, s=0.0, lx=N * h, ly=N * h)
    op = O.OracleProblem(prob)
    lv = op.levels[0]
    x = I.node_centres(N, N * h)
    X = (x - x[6])[None, :] * np.ones((N, 1))
    psi = np.broadcast_to(X ** 5, (1, lv["nd"], N, N)).copy()
    kx, ky = op.kfields(psi)
    i, j = 6, 6  # a node whose 7x7 neighbourhood is inside the domain
    Psix = 5 * X[j, i] ** 4 - 4 * h ** 4
    for n in range(lv["nd"]):
        mu = lv["mu"][n]
        Rx = -12.0 * mu * h ** 4
        cand = [h * abs(mu), 0.25 * abs(Rx) * h / (1e-3 + abs(Psix)),
                2.0 * Rx ** 2 * h / (1e-3 + abs(mu) * Psix ** 2)]
        assert abs(kx[0, n, j, i] - min(cand)) <= 1e-9 * max(cand)
        assert abs(ky[0, n, j, i]) < 1e-12  # no y variation
