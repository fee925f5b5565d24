"""Pins of the oracle's Petrov-Galerkin assembly and of its derived-field
halos, plus the committed record of how the published PG cycle behaves.
CPU only; every expected value below is a closed form or a hand-computed
number, never an oracle output.

P13  k-Diff assembly (Eqs. kxx, kyy): with k frozen to a polynomial,
     f(k psi; w) + k f(psi; w) - psi f(k; w) equals 2 (-d/dx (k dpsi/dx))
     exactly at interior nodes (the quadratic s1 is exact to degree 5, the
     mass m1 to degree 3); pg_half halves it.
P14  halos of the derived fields (Sec. 2.3 halo rule, reading R10): k and
     Psi_x copy the nearest interior node, psi follows the paper's rule
     (incoming vacuum side 0, otherwise the adjacent interior node; at a
     corner incoming in either axis gives 0).  Hand-computed values of the
     dissipation and of k_x at edge and corner nodes for a constant psi.
P15  finding: the published PG system iterated by its own cycle stagnates on
     the small two-region workload while the upwind fine scheme converges;
     the linearised cycle's spectral radius (k frozen) explains why.
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_09991_gb300 import inputs as I

# quadratic ConvFEM stencils (App. A.2), h = 1: only for writing closed forms
S1 = np.array([1 / 12, -4 / 3, 5 / 2, -4 / 3, 1 / 12])
M1 = np.array([-1 / 30, 2 / 15, 4 / 5, 2 / 15, -1 / 30])


def _dissipation(op, psi, kx, ky):
    """half (D_x + D_y) of Eq. Petrov, isolated as r(k = 0) - r(k): the other
    terms of r = b - A psi do not depend on k."""
    zero = np.zeros(op.shape)
    op.set_frozen_k(zero, zero)
    r0 = op.apply(psi)
    op.set_frozen_k(kx, ky)
    rk = op.apply(psi)
    op.set_frozen_k(None, None)
    return r0 - rk


# ---------------------------------------------------------------- P13 ----
def _poly_case(N=14, axis="x", half=0, quintic=False):
    prob = I.uniform(N, N, 4, 4, sigma_t=1.0, c=0.0, s=0.0)
    op = O.OracleProblem(prob, pg=1, pg_half=half)
    x = I.node_centres(N) - 0.5
    # psi = P(s) Q(t), k = a(s) c(t), s the axis of the dissipation
    if quintic:  # constant k: 2 K (-P'') Q exact up to degree 5 in s
        P = lambda s: 1 + s - 2 * s ** 2 + 3 * s ** 3 - s ** 4 + 2 * s ** 5
        dP = lambda s: 1 - 4 * s + 9 * s ** 2 - 4 * s ** 3 + 10 * s ** 4
        d2P = lambda s: -4 + 18 * s - 12 * s ** 2 + 40 * s ** 3
        a = lambda s: 0.03 + 0 * s
        da = lambda s: 0 * s
    else:  # quadratic k times cubic psi: k psi is quintic, exact
        P = lambda s: 1 + s - 2 * s ** 2 + 3 * s ** 3
        dP = lambda s: 1 - 4 * s + 9 * s ** 2
        d2P = lambda s: -4 + 18 * s
        a = lambda s: 0.02 + 0.01 * s + 0.03 * s ** 2
        da = lambda s: 0.01 + 0.06 * s
    Q = lambda t: 1 - t + 0.5 * t ** 2
    c = lambda t: 1 + 0.5 * t
    S, T = np.meshgrid(x, x, indexing="xy")  # S varies along columns (x)
    if axis == "y":
        S, T = T, S
    psi = np.broadcast_to(P(S) * Q(T), op.shape).copy()
    k = np.broadcast_to(a(S) * c(T), op.shape).copy()
    # 2 (-d/ds (k dpsi/ds)) = -2 c Q (a' P' + a P'')
    exact = -2.0 * c(T) * Q(T) * (da(S) * dP(S) + a(S) * d2P(S))
    if half:
        exact = 0.5 * exact
    zero = np.zeros(op.shape)
    D = _dissipation(op, psi, k, zero) if axis == "x" else _dissipation(op, psi, zero, k)
    return D, exact


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("quintic", [False, True])
def test_p13_kdiff_equals_twice_the_analytic_diffusion(axis, quintic):
    D, exact = _poly_case(axis=axis, quintic=quintic)
    inner = (slice(None), slice(None), slice(2, -2), slice(2, -2))
    err = np.abs(D[inner] - exact[None, None, 2:-2, 2:-2]).max()
    assert err < 1e-9 * np.abs(exact).max(), err


def test_p13_pg_half_halves_the_dissipation():
    D, exact = _poly_case(axis="x", half=1)
    err = np.abs(D[:, :, 2:-2, 2:-2] - exact[None, None, 2:-2, 2:-2]).max()
    assert err < 1e-9 * np.abs(exact).max(), err


# ---------------------------------------------------------------- P14 ----
def _constant_psi_case(N=12, c0=1.7):
    prob = I.uniform(N, N, 4, 4, sigma_t=1.0, c=0.0, s=0.0)  # vacuum on every side
    op = O.OracleProblem(prob, pg=1)
    lv = op.levels[0]
    h = lv["dx"]
    rng = np.random.default_rng(21)
    kcol = rng.uniform(0.01, 0.05, N)               # k(x) only
    k = np.broadcast_to(kcol[None, :], op.shape).copy()
    psi = np.full(op.shape, c0)
    D = _dissipation(op, psi, k, np.zeros(op.shape))
    return op, lv, h, kcol, c0, D


def test_p14_kdiff_halo_values_at_edges_and_corners():
    """Constant psi = c, vacuum, k = k(x) frozen, k_y = 0.  For a direction
    with mu > 0, nu > 0 (x = 0 and y = 0 incoming):
      incoming x edge (psi halo 0, k halo = k(0)):
        f(k psi) - psi f(k) = c k(0) sum_{u<0} s1_u (-1),  k f(psi) = c k(0) sum_{u>=0} s1_u
        -> D = c k(0) (5/4 + 5/4) / h^2 = 5/2 c k(0) / h^2, whatever k(1), k(2);
      outgoing x edge (everything copies, sum s1 = 0): D = 0;
      corner (0, 0), incoming in both axes (sum_{v>=0} m1_v = 9/10):
        D = c [-(1/10) S+ + (5/4)(1 + 9/10) k(0) / h^2],
        S+ = (5/2 k(0) - 4/3 k(1) + 1/12 k(2)) / h^2
        -> D = c (17/8 k(0) + 2/15 k(1) - 1/120 k(2)) / h^2;
      corner (0, N-1), y outgoing there: the incoming-x edge value;
      corner (N-1, N-1), outgoing in both: 0.
    Mirrored for mu < 0 (x = N-1 incoming)."""
    op, lv, h, k, c0, D = _constant_psi_case()
    N = op.nx
    q = lv["nd"] // 8
    rows = slice(2, N - 2)
    scale = c0 * k.max() / h ** 2
    for f in (0, 1):  # face 0: mu > 0, nu > 0; face 1: mu < 0, nu > 0
        for n in range(f * q, (f + 1) * q):
            assert (lv["mu"][n] > 0) == (f == 0) and lv["nu"][n] > 0
            Dn = D[0, n]
            xin, xout = (0, N - 1) if f == 0 else (N - 1, 0)
            sgn = 1 if f == 0 else -1
            k0, k1, k2 = k[xin], k[xin + sgn], k[xin + 2 * sgn]
            edge_in = 2.5 * c0 * k0 / h ** 2
            corner_in = c0 * (17 / 8 * k0 + 2 / 15 * k1 - 1 / 120 * k2) / h ** 2
            assert np.abs(Dn[rows, xin] - edge_in).max() < 1e-12 * scale
            assert np.abs(Dn[rows, xout]).max() < 1e-12 * scale
            assert abs(Dn[0, xin] - corner_in) < 1e-12 * scale
            assert abs(Dn[N - 1, xin] - edge_in) < 1e-12 * scale
            assert abs(Dn[N - 1, xout]) < 1e-12 * scale
            # nodes three or more columns inside see only the interior
            assert np.abs(Dn[rows, 3:N - 3]).max() < 1e-12 * scale


def test_p14_psi_x_halo_sets_k_at_the_incoming_edge():
    """k_x from the oracle's own PG coefficients (not frozen) for constant psi
    = c with mu > 0, rows far from y boundaries.  psi's zero halo at x < 0
    gives Psi_x = (7/12, -1/12, 0, ...) c / h at x = 0, 1, 2, ...; Psi_x's
    own halo copies Psi_x(0), so with m1 (moments 1, 0, 0, 0)
      (m1 * Psi_x)(0) = (9/10)(7/12) - (2/15)(1/12) = 37/72  [c / h]
      (m1 * Psi_x)(1) = (1/10)(7/12) - (4/5)(1/12)  = -1/120 [c / h]
    hence R_x = 3 mu ((m1 * Psi_x) - Psi_x) = -(5/24) mu c / h at x = 0 and
    (9/40) mu c / h at x = 1, and k_x = min{h|mu|, |R_x| h / (4 (eps + |Psi_x|)),
    2 R_x^2 h / (eps + |mu| Psi_x^2)} (Eq. ano-k, eps = 1e-3)."""
    N, c0 = 12, 1.7
    prob = I.uniform(N, N, 4, 4, sigma_t=1.0, c=0.0, s=0.0)
    op = O.OracleProblem(prob, pg=1)
    lv = op.levels[0]
    h = lv["dx"]
    kx, _ = op.kfields(np.full(op.shape, c0))
    q = lv["nd"] // 8
    psix = np.array([7 / 12, -1 / 12]) * c0 / h
    for n in range(q):  # face 0: mu > 0
        mu = lv["mu"][n]
        Rx = 3 * mu * np.array([-5 / 72, 9 / 120]) * c0 / h
        for x in (0, 1):
            cand = [h * abs(mu), 0.25 * abs(Rx[x]) * h / (1e-3 + abs(psix[x])),
                    2.0 * Rx[x] ** 2 * h / (1e-3 + abs(mu) * psix[x] ** 2)]
            assert min(cand) < cand[0]  # a branch that depends on the halos
            got = kx[0, n, 4:N - 4, x]
            assert np.abs(got - min(cand)).max() <= 1e-12 * cand[0], (n, x)
        # from x = 4 on, R_x's stencil sees only Psi_x = 0 (x >= 2)
        assert np.abs(kx[0, n, 4:N - 4, 4:]).max() < 1e-14


# ---------------------------------------------------------------- P15 ----
def test_p15_odd_even_mode_is_invisible_to_the_pg_coefficient():
    """The mechanism: d1 is odd, so f(psi; w_x) of the x-alternating mode
    (-1)^i vanishes at interior nodes (1/12 + 2/3 - 2/3 - 1/12 = 0); R_x and
    k_x vanish with it, and the central advection gives no restoring term."""
    N = 16
    prob = I.uniform(N, N, 4, 4, sigma_t=1.0, c=0.0, s=0.0, bc=(1, 1, 1, 1))
    op = O.OracleProblem(prob, pg=1)
    mode = np.broadcast_to((-1.0) ** np.arange(N)[None, :], (N, N))
    psi = np.broadcast_to(mode, op.shape).copy()
    kx, ky = op.kfields(psi)
    assert np.abs(kx[:, :, :, 4:N - 4]).max() < 1e-14
    assert np.abs(ky).max() < 1e-14


def _cycles(op, n):
    psi = op.zeros()
    hist = []
    for _ in range(n):
        psi, rel, _ = op.mg_cycle(psi)
        hist.append(rel)
    return np.array(hist)


@pytest.mark.parametrize("variant", [dict(), dict(pg_half=1), dict(beta_pg=6.0)])
def test_p15_published_pg_cycle_stagnates_on_two_region(variant):
    """32 x 32 nodes, 64 directions, two regions: 60 cycles of the PG cycle
    leave the relative residual above 0.1 (about 0.4), also with the 1/2 of
    reading R8 and with a larger Jacobi factor; the upwind fine scheme
    (pg = 0) of the same problem reaches 1e-10 within 40 cycles."""
    prob = I.two_region()
    h = _cycles(O.OracleProblem(prob, pg=1, **variant), 60)
    assert h[-10:].min() > 0.1, h[-10:]
    up = _cycles(O.OracleProblem(prob, pg=0), 40)
    assert up[-1] < 1e-10, up[-1]


def _frozen_k_spectral_radius(frac, iters=300, c=0.0):
    prob = I.uniform(8, 8, 8, 8, sigma_t=1.0, c=c, s=0.0)  # zero source: the cycle is M e
    op = O.OracleProblem(prob, pg=1)
    lv = op.levels[0]
    kx = frac * lv["dx"] * np.abs(lv["mu"])[None, :, None, None] * np.ones(op.shape)
    ky = frac * lv["dy"] * np.abs(lv["nu"])[None, :, None, None] * np.ones(op.shape)
    op.set_frozen_k(kx, ky)
    e = np.random.default_rng(1).standard_normal(op.shape)
    e /= np.linalg.norm(e)
    logs = []
    for _ in range(iters):
        e, _, _ = op.mg_cycle(e)
        n = np.linalg.norm(e)
        logs.append(np.log(n))
        e /= n
    return float(np.exp(np.mean(logs[-100:])))  # geometric mean: complex pairs too


def test_p15_frozen_k_cycle_spectral_radius():
    """Power iteration on the error propagation of the linearised cycle
    (8 x 8 nodes, 64 directions, sigma_t = 1, k frozen at a fraction of
    k_max = dx |mu|): about 0.99 for k = 0 (central ConvFEM advection alone),
    0.26 for k_max / 4, 0.48 for k_max / 2 and about 4.6 for k = k_max (the
    literal dissipation, without the 1/2, overshoots)."""
    rho = {f: _frozen_k_spectral_radius(f) for f in (0.0, 0.25, 0.5, 1.0)}
    assert 0.95 < rho[0.0] < 1.0, rho
    assert rho[0.25] < 0.35, rho
    assert 0.4 < rho[0.5] < 0.6, rho
    assert rho[1.0] > 2.0, rho
