"""ctypes wrapper of the FP64 CPU oracle (``btmg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product path never
imports this module.  It shares no code with the CUDA library; both sides
only consume the same seeded problem arrays.

Every function here marshals numpy arrays into the C oracle and back; the
arithmetic is all in ``btmg_oracle.c`` (method of arXiv 2301.09991, Sec. 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "btmg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libbtmg_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic, OpenMP over
    independent direction planes)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("lx", C.c_double), ("ly", C.c_double),
        ("order", C.c_int32),
        ("n_polar", C.c_int32), ("n_azim", C.c_int32),
        ("n_groups", C.c_int32),
        ("region", C.POINTER(C.c_int32)),
        ("n_regions", C.c_int32),
        ("sigma_t", C.POINTER(C.c_double)),
        ("sigma_s", C.POINTER(C.c_double)),
        ("source", C.POINTER(C.c_double)),
        ("bc", C.c_int32 * 4),
        ("pg", C.c_int32),
        ("nu", C.c_int32),
        ("beta_pg", C.c_double),
        ("max_levels", C.c_int32),
        ("pg_half", C.c_int32),
        ("ngauss", C.c_int32),
        ("scat_levels", C.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        dp = C.POINTER(C.c_double)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Desc)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_num_levels.argtypes = [C.c_void_p]
        L.or_level_dims.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int32), dp]
        L.or_level_quad.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp]
        L.or_level_sigt.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_level_cratio.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_get_filters.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.or_set_extra_source.argtypes = [C.c_void_p, dp]
        L.or_set_frozen_k.argtypes = [C.c_void_p, dp, dp]
        L.or_scalar_flux.argtypes = [C.c_void_p, dp, dp]
        L.or_apply.argtypes = [C.c_void_p, dp, dp]
        L.or_kfields.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_apply_planes.argtypes = [C.c_void_p, dp, C.POINTER(C.c_int32), C.c_int, dp]
        L.or_upwind_apply.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_restrict.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_prolong.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_jacobi_upwind.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, dp, C.c_int]
        L.or_pg_jacobi.argtypes = [C.c_void_p, dp, C.c_int]
        L.or_mg_cycle.restype = C.c_double
        L.or_mg_cycle.argtypes = [C.c_void_p, dp, dp]
        L.or_rel_residual.restype = C.c_double
        L.or_rel_residual.argtypes = [C.c_void_p, dp, dp]
        L.or_solve.argtypes = [C.c_void_p, dp, C.c_double, C.c_int, C.c_int, dp, dp,
                               C.c_int]
        L.or_quadrature.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
        L.or_quadrature_raw.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
        L.or_convfem_1d.argtypes = [C.c_int, dp, dp, dp, dp]
        L.or_filters_2d.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, dp, dp, dp]
        L.or_gauss01.argtypes = [C.c_int, dp, dp]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gauss01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    assert lib().or_gauss01(n, _p(x), _p(w)) == 0
    return x, w


def quadrature(nr, nc, ngauss=16, normalise=True):
    """(mu, nu, xi, p) of the 8*nr*nc octahedral directions (Sec. 2.2)."""
    nd = 8 * nr * nc
    mu, nu, xi, p = (np.zeros(nd) for _ in range(4))
    fn = lib().or_quadrature if normalise else lib().or_quadrature_raw
    assert fn(nr, nc, ngauss, _p(mu), _p(nu), _p(xi), _p(p)) == 0
    return mu, nu, xi, p


def convfem_1d(order):
    """(m1, d1, s1, m_lumped): averaged 1D ConvFEM stencils, h = 1 (Sec. 2.7)."""
    w = 2 * order + 1
    m1, d1, s1 = np.zeros(w), np.zeros(w), np.zeros(w)
    ml = np.zeros(1)
    assert lib().or_convfem_1d(order, _p(m1), _p(d1), _p(s1), _p(ml)) == 0
    return m1, d1, s1, float(ml[0])


def filters_2d(order, dx=1.0, dy=1.0):
    """dict of the 2D filters w[v, u] (v = y offset, u = x offset)."""
    w = 2 * order + 1
    arrs = [np.zeros((w, w)) for _ in range(5)]
    assert lib().or_filters_2d(order, dx, dy, *[_p(a) for a in arrs]) == 0
    return dict(zip(["wx", "wy", "wdxx", "wdyy", "wm"], arrs))


class OracleProblem:
    """A fixed-source problem held by the oracle.  ``prob`` is the dict built
    by ``paper_2301_09991_gb300.inputs`` (region map + per-region tables)."""

    def __init__(self, prob, pg=1, nu=3, beta_pg=3.0, max_levels=0, pg_half=0,
                 ngauss=16, order=None, scat_levels=0):
        self.prob = prob
        self._region = np.ascontiguousarray(prob["region"], dtype=np.int32)
        self._st = _f64(prob["sigma_t"])
        self._ss = _f64(prob["sigma_s"])
        self._src = _f64(prob["source"])
        d = _Desc()
        d.nx, d.ny = int(prob["nx"]), int(prob["ny"])
        d.lx, d.ly = float(prob["lx"]), float(prob["ly"])
        d.order = int(order if order is not None else prob.get("order", 2))
        d.n_polar, d.n_azim = int(prob["n_polar"]), int(prob["n_azim"])
        d.n_groups = int(prob["n_groups"])
        d.region = self._region.ctypes.data_as(C.POINTER(C.c_int32))
        d.n_regions = int(self._st.shape[0])
        d.sigma_t, d.sigma_s, d.source = _p(self._st), _p(self._ss), _p(self._src)
        for i, b in enumerate(prob.get("bc", (0, 0, 0, 0))):
            d.bc[i] = int(b)
        d.pg, d.nu, d.beta_pg = int(pg), int(nu), float(beta_pg)
        d.max_levels, d.pg_half, d.ngauss = int(max_levels), int(pg_half), int(ngauss)
        d.scat_levels = int(scat_levels)
        self._d = d
        self.h = lib().or_create(C.byref(d))
        if not self.h:
            raise ValueError("oracle rejected the problem description")
        self.G = d.n_groups
        self.nx, self.ny = d.nx, d.ny
        self.L = lib().or_num_levels(self.h)
        self.levels = [self.level(l) for l in range(self.L)]
        self.nd = self.levels[0]["nd"]
        self.shape = (self.G, self.nd, self.ny, self.nx)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    # -- hierarchy --------------------------------------------------------
    def level(self, l):
        dims = (C.c_int32 * 5)()
        dxdy = np.zeros(2)
        assert lib().or_level_dims(self.h, l, dims, _p(dxdy)) == 0
        nx, ny, nr, nc, nd = list(dims)
        mu, nu, xi, p = (np.zeros(nd) for _ in range(4))
        lib().or_level_quad(self.h, l, _p(mu), _p(nu), _p(xi), _p(p))
        sig = np.zeros((self._d.n_groups, ny, nx))
        lib().or_level_sigt(self.h, l, _p(sig))
        cr = np.zeros_like(sig)
        lib().or_level_cratio(self.h, l, _p(cr))
        return dict(nx=nx, ny=ny, nr=nr, nc=nc, nd=nd, dx=dxdy[0], dy=dxdy[1],
                    mu=mu, nu=nu, xi=xi, p=p, sigt=sig, cratio=cr)

    def filters(self):
        w = 2 * self._d.order + 1
        arrs = [np.zeros((w, w)) for _ in range(5)]
        lib().or_get_filters(self.h, *[_p(a) for a in arrs])
        return dict(zip(["wx", "wy", "wdxx", "wdyy", "wm"], arrs))

    # -- operators --------------------------------------------------------
    def zeros(self):
        return np.zeros(self.shape)

    def set_extra_source(self, q):
        if q is None:
            lib().or_set_extra_source(self.h, None)
        else:
            self._eq = _f64(q)
            lib().or_set_extra_source(self.h, _p(self._eq))

    def set_frozen_k(self, kx, ky):
        if kx is None:
            lib().or_set_frozen_k(self.h, None, None)
        else:
            a, b = _f64(kx), _f64(ky)
            lib().or_set_frozen_k(self.h, _p(a), _p(b))

    def scalar_flux(self, psi):
        psi = _f64(psi)
        phi = np.zeros((self.G, self.ny, self.nx))
        lib().or_scalar_flux(self.h, _p(psi), _p(phi))
        return phi

    def apply(self, psi):
        """r = b - A psi (Eq. Petrov), all groups."""
        psi = _f64(psi)
        r = np.zeros_like(psi)
        lib().or_apply(self.h, _p(psi), _p(r))
        return r

    def apply_planes(self, psi, planes):
        """Residual of selected (g, n) planes only; returns [len(planes)][ny][nx]."""
        psi = _f64(psi)
        sel = np.ascontiguousarray(np.asarray(planes, dtype=np.int32).reshape(-1))
        out = np.zeros((len(planes), self.ny, self.nx))
        lib().or_apply_planes(self.h, _p(psi), sel.ctypes.data_as(C.POINTER(C.c_int32)),
                              len(planes), _p(out))
        return out

    def kfields(self, psi):
        psi = _f64(psi)
        kx, ky = np.zeros_like(psi), np.zeros_like(psi)
        lib().or_kfields(self.h, _p(psi), _p(kx), _p(ky))
        return kx, ky

    def upwind_apply(self, l, a):
        a = _f64(a)
        out = np.zeros_like(a)
        lib().or_upwind_apply(self.h, l, _p(a), _p(out))
        return out

    def restrict(self, l, fine):
        lv = self.levels[l + 1]
        fine = _f64(fine)
        out = np.zeros((lv["nd"], lv["ny"], lv["nx"]))
        assert lib().or_restrict(self.h, l, _p(fine), _p(out)) == 0
        return out

    def prolong(self, l, coarse):
        lv = self.levels[l]
        coarse = _f64(coarse)
        out = np.zeros((lv["nd"], lv["ny"], lv["nx"]))
        assert lib().or_prolong(self.h, l, _p(coarse), _p(out)) == 0
        return out

    def jacobi_upwind(self, l, g, s, delta, sweeps):
        s = _f64(s)
        d = _f64(delta).copy()
        assert lib().or_jacobi_upwind(self.h, l, g, _p(s), _p(d), sweeps) == 0
        return d

    def pg_jacobi(self, psi, sweeps=1):
        psi = _f64(psi).copy()
        lib().or_pg_jacobi(self.h, _p(psi), sweeps)
        return psi

    def mg_cycle(self, psi):
        """One multigroup sawtooth cycle, in place on a copy.
        Returns (psi_new, rel_all, rel_per_group)."""
        psi = _f64(psi).copy()
        relg = np.zeros(self.G)
        rel = lib().or_mg_cycle(self.h, _p(psi), _p(relg))
        return psi, rel, relg

    def rel_residual(self, psi):
        psi = _f64(psi)
        relg = np.zeros(self.G)
        rel = lib().or_rel_residual(self.h, _p(psi), _p(relg))
        return rel, relg

    def solve(self, rtol=1e-8, max_cycles=500, max_outer=1, psi0=None):
        psi = self.zeros() if psi0 is None else _f64(psi0).copy()
        rel = np.zeros(1)
        hist = np.zeros(max_cycles * self.G * max(1, max_outer))
        n = lib().or_solve(self.h, _p(psi), rtol, max_cycles, max_outer, _p(rel),
                           _p(hist), hist.size)
        return psi, int(n), float(rel[0]), hist[:min(n, hist.size)]


def omp_threads():
    L = lib()
    L.or_omp_threads.restype = C.c_int
    return int(L.or_omp_threads())
