"""Seeded synthetic fixed-source problems.

This module holds no arithmetic of the method: it only draws materials and
region maps and returns plain arrays that both the CUDA library and the CPU
oracle consume.  Random numbers come from numpy's PCG64 generator
(``numpy.random.default_rng(seed)``), which gives the same stream on x86 and
Arm.

A problem is a dict with
  nx, ny, lx, ly           nodes and domain size (cell centred, dx = lx/nx)
  n_polar, n_azim          direction grid: 8 octahedron faces of
                           (n_polar/2) x (n_azim/4) patches
  n_groups                 energy groups G
  region  int32 [ny][nx]   region id of every node
  sigma_t f64 [R][G]       total cross section per region
  sigma_s f64 [R][G][G]    isotropic scattering, [to g][from g']
  source  f64 [R][G]       isotropic source per steradian
  bc      (xlo,xhi,ylo,yhi) 0 = vacuum, 1 = reflective
  order                    ConvFEM order (2 = quadratic 5x5 filters)

The workloads follow the synthetic configurations the solver is measured on
(the paper's own benchmark data, the KAIST cross sections, is not available;
its straight-duct problem of Sec. 3.1 is reproduced geometrically by
``duct``).
"""
from __future__ import annotations

import numpy as np

VACUUM, REFLECTIVE = 0, 1


def _prob(nx, ny, n_polar, n_azim, region, sigma_t, sigma_s, source, lx=1.0,
          ly=1.0, bc=(VACUUM,) * 4, order=2, name=""):
    sigma_t = np.asarray(sigma_t, dtype=np.float64)
    R, G = sigma_t.shape
    return dict(name=name, nx=int(nx), ny=int(ny), lx=float(lx), ly=float(ly),
                n_polar=int(n_polar), n_azim=int(n_azim), n_groups=int(G),
                region=np.ascontiguousarray(region, dtype=np.int32),
                sigma_t=sigma_t,
                sigma_s=np.ascontiguousarray(sigma_s, dtype=np.float64).reshape(R, G, G),
                source=np.ascontiguousarray(source, dtype=np.float64).reshape(R, G),
                bc=tuple(int(b) for b in bc), order=int(order))


def node_centres(n, length=1.0):
    """Cell-centred node coordinates x_i = (i + 1/2) dx."""
    return (np.arange(n) + 0.5) * (length / n)


def two_region(nx=32, ny=32, n_polar=8, n_azim=8, sig_in=1.0, sig_out=0.1,
               c=0.5, bc=(VACUUM,) * 4):
    """Plain one-group problem on the unit square: region 0 = the central
    quarter [0.25, 0.75]^2 with sigma_t = sig_in and source 1; region 1
    elsewhere with sigma_t = sig_out and no source; sigma_s = c sigma_t.
    (32x32 nodes, 8x8 directions is the small FP64 workload.)"""
    x = node_centres(nx)
    y = node_centres(ny)
    inside = ((x[None, :] >= 0.25) & (x[None, :] <= 0.75) &
              (y[:, None] >= 0.25) & (y[:, None] <= 0.75))
    region = np.where(inside, 0, 1)
    st = np.array([[sig_in], [sig_out]])
    ss = (c * st).reshape(2, 1, 1)
    src = np.array([[1.0], [0.0]])
    return _prob(nx, ny, n_polar, n_azim, region, st, ss, src, bc=bc,
                 name="two_region_%dx%d_%dx%d" % (nx, ny, n_polar, n_azim))


def checkerboard(n=256, n_polar=16, n_azim=32, blocks=8, seed=2, c=0.9,
                 sig_lo=0.1, sig_hi=10.0, ny=None, bc=(VACUUM,) * 4, length=1.0):
    """One-group checkerboard: blocks x blocks regions, each with its own
    sigma_t ~ logU[sig_lo, sig_hi]; sigma_s = c sigma_t; source 1 everywhere.
    (256^2 nodes, 16x32 directions, seed 2 is the FP32 single-group
    workload; ragged sizes are allowed.)  `length` is the side of the domain
    in x (the y side keeps the cell aspect ratio 1)."""
    nx = int(n)
    ny = int(ny if ny is not None else n)
    rng = np.random.default_rng(seed)
    R = blocks * blocks
    st = np.exp(rng.uniform(np.log(sig_lo), np.log(sig_hi), size=R)).reshape(R, 1)
    bx = np.minimum((np.arange(nx) * blocks) // nx, blocks - 1)
    by = np.minimum((np.arange(ny) * blocks) // ny, blocks - 1)
    region = by[:, None] * blocks + bx[None, :]
    ss = (c * st).reshape(R, 1, 1)
    src = np.ones((R, 1))
    return _prob(nx, ny, n_polar, n_azim, region, st, ss, src, bc=bc, lx=length, ly=length * ny / nx,
                 name="checkerboard_%dx%d_%dx%d_s%d" % (nx, ny, n_polar, n_azim, seed))


def multigroup(n=512, n_polar=32, n_azim=32, G=4, blocks=8, seed=3,
               absorb=0.2, sig_lo=0.1, sig_hi=10.0):
    """G-group downscatter checkerboard: per region and group
    sigma_t ~ logU[sig_lo, sig_hi]; the scattering out of group g' (a fraction
    1 - absorb of sigma_t,g') is split over the groups g >= g' by a
    Dirichlet(1,...,1) draw (lower-triangular [to][from] matrix whose column
    sums are (1-absorb) sigma_t,g'); source 1 in group 0 only.
    (512^2, 32x32 directions, G = 4, seed 3 is the mixed-precision workload.)"""
    rng = np.random.default_rng(seed)
    R = blocks * blocks
    st = np.exp(rng.uniform(np.log(sig_lo), np.log(sig_hi), size=(R, G)))
    ss = np.zeros((R, G, G))
    for r in range(R):
        for gp in range(G):
            share = rng.dirichlet(np.ones(G - gp))
            ss[r, gp:, gp] = (1.0 - absorb) * st[r, gp] * share
    bx = np.minimum((np.arange(n) * blocks) // n, blocks - 1)
    region = bx[:, None] * blocks + bx[None, :]
    src = np.zeros((R, G))
    src[:, 0] = 1.0
    return _prob(n, n, n_polar, n_azim, region, st, ss, src,
                 name="multigroup_%d_%dx%d_G%d_s%d" % (n, n_polar, n_azim, G, seed))


def voronoi(n, n_polar, n_azim, seed, k_lo=6, k_hi=20, sig_lo=0.1, sig_hi=10.0,
            c_lo=0.5, c_hi=0.95):
    """One-group Voronoi problem: K ~ U{k_lo..k_hi} sites uniform in the unit
    square; each node takes the region of its nearest site (ties to the lower
    index); sigma_t ~ logU[sig_lo, sig_hi], c ~ U[c_lo, c_hi] per region;
    source 1."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(k_lo, k_hi + 1))
    sites = rng.uniform(0.0, 1.0, size=(K, 2))
    st = np.exp(rng.uniform(np.log(sig_lo), np.log(sig_hi), size=K)).reshape(K, 1)
    c = rng.uniform(c_lo, c_hi, size=K)
    x = node_centres(n)
    X, Y = np.meshgrid(x, x)
    d2 = (X[None] - sites[:, 0, None, None]) ** 2 + (Y[None] - sites[:, 1, None, None]) ** 2
    region = np.argmin(d2, axis=0)  # argmin returns the lowest index on ties
    ss = (c.reshape(K, 1) * st).reshape(K, 1, 1)
    src = np.ones((K, 1))
    return _prob(n, n, n_polar, n_azim, region, st, ss, src,
                 name="voronoi_%d_%dx%d_s%d" % (n, n_polar, n_azim, seed))


DIRECTION_GRIDS = ((8, 16), (16, 16), (16, 32), (32, 32))


def batch(count=64, seed=4, n_lo=64, n_hi=512, step=16, grids=DIRECTION_GRIDS):
    """A batch of independent one-group Voronoi problems with uneven sizes:
    N uniform over the multiples of ``step`` in [n_lo, n_hi], direction grid
    uniform over ``grids``; problem i uses seed (seed * 1000003 + i)."""
    rng = np.random.default_rng(seed)
    sizes = np.arange(n_lo, n_hi + 1, step)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        g = grids[int(rng.integers(len(grids)))]
        out.append(voronoi(n, g[0], g[1], seed * 1000003 + i))
    return out


def duct(dx=0.8, n_polar=8, n_azim=16):
    """Straight-duct geometry of Sec. 3.1 (Fig. sing_duct_mesh, Tab.
    sing_duct_data): 28 cm x 36 cm; a 6 x 6 cm source in the centre (region 0:
    sigma_a = 0.5, S = 1); absorbers beside it in x (region 1: sigma_a = 0.5);
    6 cm wide void ducts above and below (region 2: sigma = 0); no
    scattering; vacuum boundaries."""
    lx, ly = 28.0, 36.0
    nx, ny = int(round(lx / dx)), int(round(ly / dx))
    x = node_centres(nx, lx)
    y = node_centres(ny, ly)
    in_col = (x[None, :] >= 11.0) & (x[None, :] <= 17.0)
    in_mid = (y[:, None] >= 15.0) & (y[:, None] <= 21.0)
    region = np.where(in_col & in_mid, 0, np.where(in_col, 2, 1))
    st = np.array([[0.5], [0.5], [0.0]])
    ss = np.zeros((3, 1, 1))
    src = np.array([[1.0], [0.0], [0.0]])
    return _prob(nx, ny, n_polar, n_azim, region, st, ss, src, lx=lx, ly=ly,
                 name="duct_dx%g" % dx)


def uniform(nx, ny, n_polar, n_azim, sigma_t=1.0, c=0.5, s=1.0, bc=(VACUUM,) * 4,
            lx=1.0, ly=1.0):
    """Single-region one-group problem (closed-form checks)."""
    region = np.zeros((ny, nx), dtype=np.int32)
    return _prob(nx, ny, n_polar, n_azim, region, [[sigma_t]], [[[c * sigma_t]]],
                 [[s]], lx=lx, ly=ly, bc=bc, name="uniform")


def random_field(shape, seed, lo=0.0, hi=1.0, smooth=True):
    """Seeded non-negative test field: a smooth part plus uniform noise."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(lo, hi, size=shape)
    if smooth and len(shape) >= 2:
        ny, nx = shape[-2], shape[-1]
        yy = node_centres(ny)[:, None]
        xx = node_centres(nx)[None, :]
        base = 1.0 + 0.5 * np.sin(2 * np.pi * xx) * np.cos(np.pi * yy)
        a = 0.5 * a + base
    return a
