"""Thin Python binding of the btmg C ABI (``include/btmg.h``).

Argument marshalling only: every step of the iteration runs in the CUDA
kernels of ``libbtmg.so``.  PyTorch provides device memory (caller-owned
tensors passed by ``data_ptr()``) and streams.  There is no CPU fallback: if
the library cannot be loaded or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

F64, F32, BF16, F16 = 0, 1, 2, 3
VACUUM, REFLECTIVE = 0, 1
SMOOTH_UPWIND, SMOOTH_PG = 0, 1

OK = 0
ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED = -1, -2, -3, -4
ERR_DIVERGED, ERR_TIMEOUT, ERR_NAN, ERR_UNSUPPORTED = -5, -6, -7, -8
ERR_NOALLOC_TOO_LARGE = -9

EXPORTS = (
    "btmg_create_problem", "btmg_destroy_problem", "btmg_num_unknowns", "btmg_get_layout",
    "btmg_num_levels", "btmg_level_info", "btmg_level_quadrature", "btmg_scalar_flux",
    "btmg_apply_operator", "btmg_smooth", "btmg_restrict", "btmg_prolong", "btmg_mg_cycle", "btmg_mg_cycle_host",
    "btmg_solve", "btmg_error_string", "btmg_last_error", "btmg_profile", "btmg_profile_read",
    "btmg_launch_count", "btmg_apply_operator_noalloc", "btmg_solve_refined",
    "btmg_unet_create", "btmg_unet_destroy", "btmg_unet_num_params", "btmg_unet_get_params",
    "btmg_unet_set_params", "btmg_unet_get_grads", "btmg_unet_forward", "btmg_unet_train_step",
    "btmg_unet_last_error", "btmg_set_learned", "btmg_learn_stats", "btmg_scatter_fallbacks", "btmg_convfem_stencils", "btmg_particle_balance", "btmg_learn_canvas",
    "btmg_learn_features", "btmg_create_batch", "btmg_destroy_batch", "btmg_batch_problem",
    "btmg_batch_chunks", "btmg_batch_coarse", "btmg_batch_wait_selftest", "btmg_solve_batch", "btmg_wait_selftest", "btmg_fp32_fma_rate",
)
LEARN_FEATURES = 4  # input channels of the learned correction
PROF_CLASSES = ("pg_residual", "pg_jacobi", "upwind_fine", "upwind_coarse", "restrict", "misc")


class Desc(C.Structure):
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
        ("nu_jacobi", C.c_int32),
        ("beta_pg", C.c_double),
        ("psi_dtype", C.c_int32),
        ("max_levels", C.c_int32),
        ("pg_half", C.c_int32),
        ("chunks", C.c_int32),
        ("scat_levels", C.c_int32),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("cycles", C.c_int32), ("status", C.c_int32), ("rel_resid", C.c_double),
        ("history", C.POINTER(C.c_double)), ("history_len", C.c_int32),
        ("check_every", C.c_int32), ("max_outer", C.c_int32),
    ]


class BtmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("btmg error %d (%s): %s" % (code, error_string(code), msg))
        self.code = code


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``libbtmg.so`` (building it in-tree if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError("libbtmg.so is not built: run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(path)
    vp, i32, i64p = C.c_void_p, C.c_int32, C.POINTER(C.c_int64)
    dp = C.POINTER(C.c_double)
    L.btmg_create_problem.argtypes = [C.POINTER(Desc), vp, C.POINTER(vp)]
    L.btmg_destroy_problem.argtypes = [vp]
    L.btmg_num_unknowns.argtypes = [vp, i64p]
    L.btmg_get_layout.argtypes = [vp, i64p]
    L.btmg_num_levels.argtypes = [vp, C.POINTER(i32)]
    L.btmg_level_info.argtypes = [vp, i32, C.POINTER(i32), dp]
    L.btmg_level_quadrature.argtypes = [vp, i32, dp, dp, dp]
    L.btmg_scalar_flux.argtypes = [vp, vp, vp, vp]
    L.btmg_apply_operator.argtypes = [vp, vp, vp, vp]
    L.btmg_smooth.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp]
    L.btmg_restrict.argtypes = [vp, i32, vp, vp, vp]
    L.btmg_prolong.argtypes = [vp, i32, vp, vp, vp]
    L.btmg_mg_cycle.argtypes = [vp, vp, dp, vp]
    L.btmg_mg_cycle_host.argtypes = [vp, vp, vp, dp, vp]
    L.btmg_solve.argtypes = [vp, vp, C.c_double, i32, C.POINTER(SolveInfo), vp]
    L.btmg_profile.argtypes = [vp, i32]
    L.btmg_profile_read.argtypes = [vp, dp, i64p, i32]
    L.btmg_launch_count.argtypes = [vp, i64p]
    L.btmg_solve_refined.argtypes = [vp, vp, C.c_double, i32, i32, C.POINTER(SolveInfo), vp]
    L.btmg_apply_operator_noalloc.argtypes = [i32, i32, C.c_double, C.c_double, i32, i32,
                                              C.POINTER(i32), i32, i32, vp, vp, vp, vp, vp, vp, dp]
    L.btmg_set_learned.argtypes = [vp, vp, i32]
    L.btmg_learn_stats.argtypes = [vp, i64p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(i32)]
    L.btmg_scatter_fallbacks.argtypes = [vp, C.POINTER(i32)]
    L.btmg_particle_balance.argtypes = [vp, vp, C.POINTER(C.c_double), vp]
    L.btmg_convfem_stencils.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
    L.btmg_learn_canvas.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    L.btmg_learn_features.argtypes = [vp, vp, vp, vp, vp, vp]
    L.btmg_wait_selftest.argtypes = [i32, vp]
    L.btmg_fp32_fma_rate.argtypes = [i32, dp, vp]
    L.btmg_create_batch.argtypes = [C.POINTER(Desc), i32, i32, vp, C.POINTER(vp)]
    L.btmg_destroy_batch.argtypes = [vp]
    L.btmg_batch_problem.argtypes = [vp, i32, C.POINTER(vp)]
    L.btmg_batch_chunks.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), dp]
    L.btmg_batch_coarse.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), dp]
    L.btmg_batch_wait_selftest.argtypes = [vp]
    L.btmg_solve_batch.argtypes = [vp, C.POINTER(vp), C.c_double, i32, i32, C.POINTER(SolveInfo), vp]
    L.btmg_unet_create.argtypes = [i32, C.c_uint64, C.POINTER(vp)]
    L.btmg_unet_destroy.argtypes = [vp]
    L.btmg_unet_num_params.argtypes = [vp, i64p]
    fp = C.POINTER(C.c_float)
    L.btmg_unet_get_params.argtypes = [vp, fp, C.c_int64]
    L.btmg_unet_set_params.argtypes = [vp, fp, C.c_int64]
    L.btmg_unet_get_grads.argtypes = [vp, fp, C.c_int64]
    L.btmg_unet_forward.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    L.btmg_unet_train_step.argtypes = [vp, vp, vp, i32, i32, i32, C.c_float, dp, vp]
    L.btmg_unet_last_error.restype = C.c_char_p
    L.btmg_error_string.restype = C.c_char_p
    L.btmg_error_string.argtypes = [C.c_int]
    L.btmg_last_error.restype = C.c_char_p
    L.btmg_last_error.argtypes = []
    _lib = L
    return L


def fp32_fma_rate(repeats=5, stream=None):
    """Measured FP32 FMA throughput of this GPU (TFLOP/s)."""
    t = C.c_double()
    _check(load().btmg_fp32_fma_rate(int(repeats), C.byref(t), _stream_ptr(stream)))
    return t.value


def wait_selftest(polls=1000, stream=None):
    """Run the bounded-wait failure path once; returns the status code
    (ERR_TIMEOUT expected)."""
    return load().btmg_wait_selftest(int(polls), _stream_ptr(stream))


def error_string(code):
    return load().btmg_error_string(int(code)).decode()


def _check(rc):
    if rc != OK:
        raise BtmgError(rc, load().btmg_last_error().decode())
    return rc


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype_of(code):
    torch = _torch()
    return {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}[code]


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def make_desc(prob, dtype=F32, pg=1, nu=3, beta_pg=3.0, max_levels=0, pg_half=0, order=None, chunks=0,
              scat_levels=0):
    """btmg_problem_desc of a problem dict (see inputs.py) and the host arrays
    it points to (keep them alive until the problem is created)."""
    keep = (np.ascontiguousarray(prob["region"], dtype=np.int32),
            np.ascontiguousarray(prob["sigma_t"], dtype=np.float64),
            np.ascontiguousarray(prob["sigma_s"], dtype=np.float64),
            np.ascontiguousarray(prob["source"], dtype=np.float64))
    region, st, ss, src = keep
    d = Desc()
    d.nx, d.ny = int(prob["nx"]), int(prob["ny"])
    d.lx, d.ly = float(prob["lx"]), float(prob["ly"])
    d.order = int(order if order is not None else prob.get("order", 2))
    d.n_polar, d.n_azim = int(prob["n_polar"]), int(prob["n_azim"])
    d.n_groups = int(st.shape[1])
    d.region = region.ctypes.data_as(C.POINTER(C.c_int32))
    d.n_regions = int(st.shape[0])
    dp = C.POINTER(C.c_double)
    d.sigma_t = st.ctypes.data_as(dp)
    d.sigma_s = ss.ctypes.data_as(dp)
    d.source = src.ctypes.data_as(dp)
    for i, b in enumerate(prob.get("bc", (0, 0, 0, 0))):
        d.bc[i] = int(b)
    d.pg, d.nu_jacobi, d.beta_pg = int(pg), int(nu), float(beta_pg)
    d.psi_dtype, d.max_levels, d.pg_half = int(dtype), int(max_levels), int(pg_half)
    d.chunks = int(chunks)
    d.scat_levels = int(scat_levels)
    return d, keep


def convfem_stencils(order):
    """(m1, d1, s1) ConvFEM 1D stencils of the order at offsets -3..3, as the
    library derives them (host computation, no device needed)."""
    arrs = [np.zeros(7) for _ in range(3)]
    _check(load().btmg_convfem_stencils(int(order), *[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs]))
    return tuple(arrs)


class Problem:
    """A fixed-source problem resident on the GPU.

    ``prob`` is a dict of plain arrays (see ``inputs.py``): nx, ny, lx, ly,
    n_polar, n_azim, region [ny][nx], sigma_t [R][G], sigma_s [R][G][G],
    source [R][G], bc.  ``dtype`` is the storage type of psi.
    """

    def __init__(self, prob, dtype=F32, pg=1, nu=3, beta_pg=3.0, max_levels=0, pg_half=0,
                 order=None, stream=None, chunks=0, scat_levels=0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("btmg needs a CUDA device (sm_103a); there is no CPU path")
        L = load()
        d, self._keep = make_desc(prob, dtype, pg, nu, beta_pg, max_levels, pg_half, order, chunks, scat_levels)
        h = C.c_void_p()
        _check(L.btmg_create_problem(C.byref(d), _stream_ptr(stream), C.byref(h)))
        self._owned = True
        self._attach(h, d)

    @classmethod
    def _view(cls, h, d, owner):
        """A problem owned by a Batch (not destroyed by this object)."""
        self = cls.__new__(cls)
        self._owned = False
        self._owner = owner
        self._attach(h, d)
        return self

    def _attach(self, h, d):
        torch = _torch()
        L = load()
        self.desc = d
        self.h = h
        self.dtype_code = int(d.psi_dtype)
        self.torch_dtype = _dtype_of(self.dtype_code)
        self.compute_dtype = torch.float64 if self.dtype_code == F64 else torch.float32
        self.G = d.n_groups
        n = C.c_int32()
        _check(L.btmg_num_levels(self.h, C.byref(n)))
        self.L = n.value
        self.levels = [self.level_info(l) for l in range(self.L)]
        self.nd = self.levels[0]["nd"]
        self.shape = (self.G, self.nd, d.ny, d.nx)

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            load().btmg_destroy_problem(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries -------------------------------------------------------------
    def num_unknowns(self):
        n = C.c_int64()
        _check(load().btmg_num_unknowns(self.h, C.byref(n)))
        return n.value

    def layout(self):
        s = (C.c_int64 * 6)()
        _check(load().btmg_get_layout(self.h, s))
        return tuple(s)

    def level_info(self, l):
        dims = (C.c_int32 * 5)()
        dxdy = (C.c_double * 2)()
        _check(load().btmg_level_info(self.h, l, dims, dxdy))
        nd = dims[4]
        mu, nu, w = np.zeros(nd), np.zeros(nd), np.zeros(nd)
        dp = C.POINTER(C.c_double)
        _check(load().btmg_level_quadrature(self.h, l, mu.ctypes.data_as(dp), nu.ctypes.data_as(dp),
                                            w.ctypes.data_as(dp)))
        return dict(nx=dims[0], ny=dims[1], nr=dims[2], nc=dims[3], nd=nd, dx=dxdy[0], dy=dxdy[1],
                    mu=mu, nu=nu, p=w)

    def level_shape(self, l):
        lv = self.levels[l]
        return (lv["nd"], lv["ny"], lv["nx"])

    def solve_refined(self, psi64, rtol=1e-10, max_outer=60, inner_cycles=4, stream=None):
        """Mixed-precision solve: FP64 outer residual, inner cycles in this
        problem's storage type.  psi64: contiguous CUDA float64 tensor."""
        torch = _torch()
        if not (psi64.is_cuda and psi64.dtype == torch.float64 and psi64.is_contiguous()
                and tuple(psi64.shape) == self.shape):
            raise ValueError("psi64 must be a contiguous CUDA float64 tensor %s" % (self.shape,))
        info = SolveInfo()
        hist = np.zeros(max_outer + 1)
        info.history = hist.ctypes.data_as(C.POINTER(C.c_double))
        info.history_len = hist.size
        rc = load().btmg_solve_refined(self.h, _ptr(psi64), float(rtol), int(max_outer), int(inner_cycles),
                                       C.byref(info), _stream_ptr(stream))
        if rc not in (OK, ERR_NOT_CONVERGED):
            _check(rc)
        n_outer = int(np.count_nonzero(hist)) if info.rel_resid > 0 else 1
        return dict(status=rc, cycles=info.cycles, rel_resid=info.rel_resid, history=hist[:max(n_outer, 1)].copy())

    def set_learned(self, unet, every=1):
        """Attach (or with None detach) a learned correction, see btmg.h."""
        self._unet = unet  # keep the network alive while attached
        _check(load().btmg_set_learned(self.h, unet.h if unet is not None else None, int(every)))

    def particle_balance(self, psi, stream=None):
        """Per group (production, removal, leakage, relative imbalance) of psi
        for the upwind fine scheme (btmg_particle_balance); [G][4] array."""
        self._check_psi(psi)
        out = np.zeros(4 * self.G)
        _check(load().btmg_particle_balance(self.h, _ptr(psi), out.ctypes.data_as(C.POINTER(C.c_double)),
                                            _stream_ptr(stream)))
        return out.reshape(self.G, 4)

    def scatter_fallbacks(self):
        """Solves on this problem that dropped the scattering smoother
        (fallback arbitrated by plain multigrid)."""
        n = C.c_int32()
        _check(load().btmg_scatter_fallbacks(self.h, C.byref(n)))
        return n.value

    def learn_stats(self):
        """(learned steps, mean residual reduction factor, last alpha,
        solves that fell back to plain cycles)."""
        n, f, a, b = C.c_int64(), C.c_double(), C.c_double(), C.c_int32()
        _check(load().btmg_learn_stats(self.h, C.byref(n), C.byref(f), C.byref(a), C.byref(b)))
        return n.value, f.value, a.value, b.value

    def learn_canvas(self):
        """(H8, W8, f): coarse canvas of the learned correction and its factor."""
        h8, w8, f = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().btmg_learn_canvas(self.h, C.byref(h8), C.byref(w8), C.byref(f)))
        return h8.value, w8.value, f.value

    def learn_features(self, psi, psi_prev=None, stream=None):
        """(features [G][H8][W8][4], scale [G]) of the learned step for psi
        (psi_prev: the iterate one cycle earlier, or None)."""
        torch = _torch()
        h8, w8, _ = self.learn_canvas()
        feat = torch.empty((self.G, h8, w8, LEARN_FEATURES), dtype=torch.float32, device="cuda")
        scale = torch.empty((self.G,), dtype=torch.float32, device="cuda")
        prev = _ptr(psi_prev) if psi_prev is not None else None
        _check(load().btmg_learn_features(self.h, _ptr(psi), prev, _ptr(feat), _ptr(scale), _stream_ptr(stream)))
        return feat, scale

    def profile(self, enable=True):
        _check(load().btmg_profile(self.h, int(bool(enable))))

    def profile_read(self):
        n = len(PROF_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        _check(load().btmg_profile_read(self.h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(PROF_CLASSES)}

    def launch_count(self):
        n = C.c_int64()
        _check(load().btmg_launch_count(self.h, C.byref(n)))
        return n.value

    # -- buffers -------------------------------------------------------------
    def zeros(self):
        return _torch().zeros(self.shape, dtype=self.torch_dtype, device="cuda")

    def _check_psi(self, psi):
        torch = _torch()
        if not (psi.is_cuda and psi.dtype == self.torch_dtype and psi.is_contiguous()
                and tuple(psi.shape) == self.shape):
            raise ValueError("psi must be a contiguous CUDA tensor %s of %s" % (self.shape, self.torch_dtype))

    # -- operations (names follow the C ABI) ---------------------------------
    def scalar_flux(self, psi, stream=None):
        self._check_psi(psi)
        phi = _torch().empty((self.G, self.shape[2], self.shape[3]), dtype=self.compute_dtype, device="cuda")
        _check(load().btmg_scalar_flux(self.h, _ptr(psi), _ptr(phi), _stream_ptr(stream)))
        return phi

    def apply_operator(self, psi, r=None, stream=None):
        self._check_psi(psi)
        if r is None:
            r = _torch().empty(self.shape, dtype=self.compute_dtype, device="cuda")
        _check(load().btmg_apply_operator(self.h, _ptr(psi), _ptr(r), _stream_ptr(stream)))
        return r

    def smooth_pg(self, psi, sweeps=1, stream=None):
        self._check_psi(psi)
        _check(load().btmg_smooth(self.h, _ptr(psi), None, 0, 0, sweeps, SMOOTH_PG, _stream_ptr(stream)))
        return psi

    def smooth_upwind(self, delta, src, level, group=0, sweeps=3, stream=None):
        shp = self.level_shape(level)
        for t in (delta, src):
            if tuple(t.shape) != shp or t.dtype != self.compute_dtype or not t.is_cuda:
                raise ValueError("level %d buffers must be %s %s" % (level, shp, self.compute_dtype))
        _check(load().btmg_smooth(self.h, _ptr(delta), _ptr(src), level, group, sweeps, SMOOTH_UPWIND,
                                  _stream_ptr(stream)))
        return delta

    def restrict(self, level, fine, stream=None):
        coarse = _torch().empty(self.level_shape(level + 1), dtype=self.compute_dtype, device="cuda")
        _check(load().btmg_restrict(self.h, level, _ptr(fine), _ptr(coarse), _stream_ptr(stream)))
        return coarse

    def prolong(self, level, coarse, stream=None):
        fine = _torch().empty(self.level_shape(level), dtype=self.compute_dtype, device="cuda")
        _check(load().btmg_prolong(self.h, level, _ptr(coarse), _ptr(fine), _stream_ptr(stream)))
        return fine

    def mg_cycle(self, psi, want_residual=True, stream=None):
        self._check_psi(psi)
        rel = C.c_double(0.0)
        _check(load().btmg_mg_cycle(self.h, _ptr(psi), C.byref(rel) if want_residual else None,
                                    _stream_ptr(stream)))
        return rel.value if want_residual else None

    def mg_cycle_host(self, psi_in, psi_out=None, want_residual=True, stream=None):
        """One cycle on host tensors (btmg_mg_cycle_host): psi_in, psi_out
        contiguous CPU tensors of the problem's shape and storage type
        (psi_out defaults to psi_in; page-locked memory lets the copy back
        overlap the last kernel).  Returns the relative residual of the
        input, or None."""
        psi_out = psi_in if psi_out is None else psi_out
        for t in (psi_in, psi_out):
            if t.is_cuda or t.dtype != self.torch_dtype or not t.is_contiguous() or tuple(t.shape) != self.shape:
                raise ValueError("psi_in/psi_out must be contiguous CPU tensors %s of %s" % (self.shape, self.torch_dtype))
        rel = C.c_double(0.0)
        _check(load().btmg_mg_cycle_host(self.h, _ptr(psi_in), _ptr(psi_out),
                                         C.byref(rel) if want_residual else None, _stream_ptr(stream)))
        return rel.value if want_residual else None

    def solve(self, psi, rtol=1e-6, max_cycles=1000, check_every=1, max_outer=0, history=True,
              stream=None, raise_on_fail=False):
        self._check_psi(psi)
        info = SolveInfo()
        hist = np.zeros(max_cycles * self.G * max(1, max_outer or 8)) if history else None
        if hist is not None:
            info.history = hist.ctypes.data_as(C.POINTER(C.c_double))
            info.history_len = hist.size
        info.check_every = int(check_every)
        info.max_outer = int(max_outer)
        rc = load().btmg_solve(self.h, _ptr(psi), float(rtol), int(max_cycles), C.byref(info),
                               _stream_ptr(stream))
        if rc not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_NAN) or (raise_on_fail and rc != OK):
            _check(rc)
        out = dict(status=rc, cycles=info.cycles, rel_resid=info.rel_resid)
        if hist is not None:
            out["history"] = hist[:min(info.cycles, hist.size)].copy()
        return out


class Batch:
    """Independent problems solved together (btmg_create_batch /
    btmg_solve_batch): one graph launch advances every unconverged problem
    by one cycle.  `problems[i]` are non-owning Problem views."""

    def __init__(self, probs, dtype=F32, pg=0, nu=3, autotune=False, chunks=None, stream=None, scat_levels=0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("btmg needs a CUDA device (sm_103a); there is no CPU path")
        L = load()
        n = len(probs)
        descs = (Desc * n)()
        self._keep = []
        for i, prob in enumerate(probs):
            d, keep = make_desc(prob, dtype, pg, nu, chunks=(chunks[i] if chunks else 0), scat_levels=scat_levels)
            descs[i] = d
            self._keep.append(keep)
        h = C.c_void_p()
        _check(L.btmg_create_batch(descs, n, int(bool(autotune)), _stream_ptr(stream), C.byref(h)))
        self.h = h
        self.problems = []
        for i in range(n):
            ph = C.c_void_p()
            _check(L.btmg_batch_problem(self.h, i, C.byref(ph)))
            self.problems.append(Problem._view(ph, descs[i], self))

    def chunks(self, i):
        """(chunks, automatic chunks, tuned ms per eager cycle) of problem i."""
        c, a, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(load().btmg_batch_chunks(self.h, i, C.byref(c), C.byref(a), C.byref(ms)))
        return c.value, a.value, ms.value

    def coarse(self):
        """(persistent, tile width, CTAs per SM, tuned ms per launch) of the
        batch's persistent coarse-correction launch."""
        p, t, c, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        _check(load().btmg_batch_coarse(self.h, C.byref(p), C.byref(t), C.byref(c), C.byref(ms)))
        return bool(p.value), t.value, c.value, ms.value

    def zeros(self):
        return [p.zeros() for p in self.problems]

    def solve(self, psis, rtol=1e-6, max_cycles=1000, check_every=1, stream=None):
        """Solve every problem from psis[i] (device tensors, in place); returns
        (status, [dict(status, cycles, rel_resid)])."""
        n = len(self.problems)
        if len(psis) != n:
            raise ValueError("need one psi per problem")
        for p, x in zip(self.problems, psis):
            p._check_psi(x)
        ptrs = (C.c_void_p * n)(*[x.data_ptr() for x in psis])
        infos = (SolveInfo * n)()
        rc = load().btmg_solve_batch(self.h, ptrs, float(rtol), int(max_cycles), int(check_every), infos,
                                     _stream_ptr(stream))
        if rc not in (OK, ERR_NOT_CONVERGED):
            _check(rc)
        return rc, [dict(status=infos[i].status, cycles=infos[i].cycles, rel_resid=infos[i].rel_resid)
                    for i in range(n)]

    def close(self):
        if getattr(self, "h", None):
            for p in self.problems:
                p.h = None
            load().btmg_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ucheck(rc):
    if rc != OK:
        raise BtmgError(rc, load().btmg_unet_last_error().decode())


class UNet:
    """The learned-correction U-net held on the GPU (see btmg.h)."""

    def __init__(self, in_channels=3, seed=1):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("btmg needs a CUDA device (sm_103a); there is no CPU path")
        h = C.c_void_p()
        _ucheck(load().btmg_unet_create(int(in_channels), int(seed), C.byref(h)))
        self.h = h
        self.in_channels = in_channels
        n = C.c_int64()
        _ucheck(load().btmg_unet_num_params(self.h, C.byref(n)))
        self.nparam = n.value

    def close(self):
        if getattr(self, "h", None):
            load().btmg_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        a = np.zeros(self.nparam, dtype=np.float32)
        _ucheck(load().btmg_unet_get_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), self.nparam))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        _ucheck(load().btmg_unet_set_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), self.nparam))

    def get_grads(self):
        a = np.zeros(self.nparam, dtype=np.float32)
        _ucheck(load().btmg_unet_get_grads(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), self.nparam))
        return a

    def forward(self, x, stream=None):
        """x: CUDA float32 [N][H][W][in_channels] -> CUDA float32 [N][H][W]."""
        n, h, w, c = x.shape
        y = _torch().empty((n, h, w), dtype=_torch().float32, device="cuda")
        _ucheck(load().btmg_unet_forward(self.h, _ptr(x.contiguous()), _ptr(y), n, h, w, _stream_ptr(stream)))
        return y

    def train_step(self, x, target, lr, want_loss=True, stream=None):
        n, h, w, c = x.shape
        loss = C.c_double(0.0)
        _ucheck(load().btmg_unet_train_step(self.h, _ptr(x.contiguous()), _ptr(target.contiguous()), n, h, w,
                                            float(lr), C.byref(loss) if want_loss else None,
                                            _stream_ptr(stream)))
        return loss.value if want_loss else None
