// k_mg_impl.cuh -- the HBM-bound multigrid kernels (instantiated per
// storage type in k_mg_f64.cu, k_mg_f32.cu and k_mg_lp.cu):
//   * upwind Jacobi (Eq. matrix_full with beta = 1, upwind filters of
//     Sec. 2.4), nu sweeps temporally blocked in one pass: a 32x32 output
//     tile loads its source and initial correction on the tile extended by
//     nu nodes on the two upwind sides, sweeps in shared memory (the
//     upwind stencil only reaches one node upstream per sweep), and writes
//     the result once.  UpSamp (Sec. 2.5) of the coarser correction is
//     fused into the load; on the finest level the update psi += delta and
//     the scalar-flux partial sums are fused into the store.
//   * restriction (Sec. 2.5): coarse = sum_children p dx dy fine / (P dX dY)
//   * UpSamp prolongation, scalar-flux partials, source assembly and a
//     deterministic FP64 sum.
#pragma once
#include <cstring>
#include <type_traits>

#include "btmg_common.cuh"
#include "tma.cuh"

namespace btmg {
namespace {

constexpr int UT = 32, UNT = 256, NUMAX = 8;

// Region of one direction: the 32x32 output tile extended by NU nodes on the
// two upwind sides (W x W), stored with a one-cell zero ring (stride W + 2).
// Region cell i is owned by thread i mod 256 (slot i / 256): the same cells
// for every direction, so the next direction's inputs are fetched into
// registers while the current one sweeps, and each cell keeps its source and
// inverse diagonal in registers.
//
// A sweep updates every owned cell without validity checks: after k sweeps
// only the cells at least k cells downwind of the region's upwind edge are
// exact, and the output tile is exactly the set that is exact after NU
// sweeps.  Cells outside the domain get source 0 and inverse diagonal 0, so
// they stay 0 (the vacuum halo); on a reflective incoming side the cell next
// to the boundary is re-copied after every sweep.
// FP32: the fast reciprocal (2 ulp, the Jacobi diagonal tolerates it); FP64: exact
__device__ __forceinline__ float rcp_(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double rcp_(double v) { return 1.0 / v; }
// shared bytes of one tile of width TU with NU sweeps (two sweep buffers
// with their zero ring and spare cell, and the sigma region)
template <typename C, int NU, int TU> constexpr size_t upwind_smem() {
  return (2 * ((size_t)(TU + NU + 2) * (TU + NU + 2) + 1) + (size_t)(TU + 2 * NU) * (TU + 2 * NU)) * sizeof(C);
}
// One TU x TU tile (tile index `tile` of a grid tiles_x wide) and direction
// chunk `chunk` of the nu-sweep upwind Jacobi, by the 256 threads of a CTA;
// smem_raw holds upwind_smem<C, NU, TU>() bytes.
template <typename T, typename C, int MODE, int NU, int TU>
__device__ __forceinline__ void upwind_tile(const UpArgs<T, C>& a, const int tile, const int chunk,
                                            unsigned char* smem_raw) {
  static_assert(TU * TU % UNT == 0 && UNT % TU == 0, "tile rows per thread");
  constexpr int RPT = TU * TU / UNT, RSTEP = UNT / TU;  // tile rows per thread, row step
  constexpr int W = TU + NU;        // loaded region (tile + NU upwind nodes)
  constexpr int WP = W + 2;         // stride with the zero ring
  constexpr int WS = TU + 2 * NU;   // sigma region covering both upwind sides
  constexpr int NS = (W * W + UNT - 1) / UNT;  // region cells per thread
  // two sweep buffers, each followed by one spare cell that the unused
  // slots of the last thread row read and write (no per-cell tests)
  constexpr int DB = WP * WP + 1;
  C* D0 = reinterpret_cast<C*>(smem_raw);
  C* D1 = D0 + DB;
  C* SG = D1 + DB;

  const int tid = threadIdx.x, tx = tid % TU, ty = tid / TU;
  const int x0 = (tile % a.tiles_x) * TU, y0 = (tile / a.tiles_x) * TU;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;

  for (int i = tid; i < WS * WS; i += UNT) {
    const int gx = x0 - NU + i % WS, gy = y0 - NU + i / WS;
    SG[i] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? a.sig[gy * nx + gx] : C(0);
  }
  for (int i = tid; i < 2 * DB; i += UNT) D0[i] = C(0);  // zero rings of D0 and D1

  // The region's placement depends only on the signs of mu and nu, which a
  // chunk of directions (inside one octant face) shares: the global offset
  // of each owned cell (-1 outside the domain), its UpSamp parent offset and
  // its sigma are computed once per sign combination, not per direction.
  int gofs[NS], cofs[NS];
  C sgv[NS];
  // byte offset into a sweep buffer of each slot's cell (one-cell ring
  // around the region), or of the spare cell for an unused slot (whose
  // upstream reads stay inside the shared allocation and are never used)
  unsigned cb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int i = tid + UNT * s;
    cb[s] = (unsigned)(i < W * W ? (i / W + 1) * WP + i % W + 1 : WP * WP) * sizeof(C);
  }
  int combo = -1;
  const int shx = a.fx >> 1, shy = a.fy >> 1;
  auto geom = [&](int cmb) {
    const bool sxp = cmb & 1, syp = cmb & 2;
    const int ox = x0 - (sxp ? NU : 0), oy = y0 - (syp ? NU : 0);
    const int sgx = sxp ? 0 : NU, sgy = syp ? 0 : NU;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = tid + UNT * s;
      const int ly = i / W, lx = i % W;
      const int gx = ox + lx, gy = oy + ly;
      const bool in = i < W * W && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
      gofs[s] = in ? gy * nx + gx : -1;
      cofs[s] = in ? (gy >> shy) * a.nxc + (gx >> shx) : 0;
      sgv[s] = in ? SG[(ly + sgy) * WS + lx + sgx] : C(0);
    }
    combo = cmb;
  };

  C phi_acc[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) phi_acc[k] = C(0);

  const int n_begin = chunk * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);

  // registers holding the next direction's inputs
  C rs[NS], rd[NS], rp[RPT];
  // this thread's tile nodes (column tx, rows ty + RSTEP k): offset of row 0
  // and the rows inside the domain
  const int pofs = (y0 + ty) * nx + x0 + tx;
  int pmask = 0;
#pragma unroll
  for (int k = 0; k < RPT; ++k)
    if (x0 + tx < nx && y0 + ty + RSTEP * k < ny) pmask |= 1 << k;
  auto fetch = [&](int n) {
    const Dir<C> dr = a.dir[n];
    const int cmb = (dr.mu > C(0) ? 1 : 0) | (dr.nu > C(0) ? 2 : 0);
    if (cmb != combo) geom(cmb);  // after the current direction's set-up
    const C* srcn = a.src + (size_t)n * a.src_stride;
    const C* initn = a.init_mode == INIT_UPSAMPLE ? a.init + (size_t)a.parent[n] * ((size_t)a.nyc * a.nxc)
                                                  : a.init + (size_t)n * npix;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      C v = C(0), d = C(0);
      if (gofs[s] >= 0) {
        v = srcn[gofs[s]];
        if (a.init_mode == INIT_UPSAMPLE)
          d = initn[cofs[s]];
        else if (a.init_mode == INIT_SAME)
          d = initn[gofs[s]];
      }
      rs[s] = v;
      rd[s] = d;
    }
    if (MODE == UP_UPDATE) {
      const T* pin_n = a.psi_in + (size_t)n * npix + pofs;
#pragma unroll
      for (int k = 0; k < RPT; ++k) rp[k] = (pmask >> k) & 1 ? (C)Conv<T>::ld(pin_n + RSTEP * k * nx) : C(0);
    }
  };

  __syncthreads();  // SG is complete before the first geometry reads it
  if (n_begin < n_end) fetch(n_begin);
  // Each direction writes its initial correction into the buffer that does
  // not hold the previous direction's result: the last reads of that buffer
  // were in the previous direction's final sweep, which ended at a barrier,
  // so no barrier is needed before the write.
  // With nu odd the result of a direction lands in D1 and the next one
  // starts from D0 again: the buffers stay fixed (constant offsets).
  C* Dinit = D0;
  C* Dother = D1;
  auto at = [](C* D, unsigned off) -> C& { return *reinterpret_cast<C*>(reinterpret_cast<char*>(D) + off); };

  for (int n = n_begin; n < n_end; ++n) {
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    const int ox = x0 - (sxp ? NU : 0), oy = y0 - (syp ? NU : 0);
    const C ax = dr.ax, ay = dr.ay, axy = dr.ax + dr.ay;
    // this direction's upstream cells as byte offsets (register + constant
    // buffer offset in the sweeps)
    unsigned ofx[NS], ofy[NS];
    {
      const unsigned ub = sxp ? (unsigned)-(int)sizeof(C) : (unsigned)sizeof(C);
      const unsigned vb = syp ? (unsigned)(-WP * (int)sizeof(C)) : (unsigned)(WP * sizeof(C));
#pragma unroll
      for (int s = 0; s < NS; ++s) ofx[s] = cb[s] + ub, ofy[s] = cb[s] + vb;
    }
    // reflective incoming sides touching this region: column / row to re-copy
    const bool rx_ = sxp ? (a.bc.xlo == BC_REFLECTIVE && ox < 0) : (a.bc.xhi == BC_REFLECTIVE && ox + W > nx);
    const bool ry_ = syp ? (a.bc.ylo == BC_REFLECTIVE && oy < 0) : (a.bc.yhi == BC_REFLECTIVE && oy + W > ny);
    const int bxl = sxp ? -ox : nx - 1 - ox;  // local column of the boundary node
    const int byl = syp ? -oy : ny - 1 - oy;
    const int hxl = sxp ? bxl - 1 : bxl + 1;  // its upwind halo cell
    const int hyl = syp ? byl - 1 : byl + 1;
    C sreg[NS], ireg[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {  // the geometry of this direction's signs (set by its fetch)
      sreg[s] = rs[s];
      ireg[s] = gofs[s] >= 0 ? rcp_(axy + sgv[s]) : C(0);
      at(Dinit, cb[s]) = rd[s];
    }
    C pin[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) pin[k] = rp[k];
    if (n + 1 < n_end) fetch(n + 1);  // in flight during the sweeps
    __syncthreads();
    C* Dold = Dinit;
    C* Dnew = Dother;
    auto recopy = [&](C* D) {  // reflective halo = adjacent interior node
      if (rx_)
        for (int ly = tid; ly < W; ly += UNT)
          if (hxl >= 0 && hxl < W && bxl >= 0 && bxl < W) D[(ly + 1) * WP + hxl + 1] = D[(ly + 1) * WP + bxl + 1];
      if (ry_)
        for (int lx = tid; lx < W; lx += UNT)
          if (hyl >= 0 && hyl < W && byl >= 0 && byl < W) D[(hyl + 1) * WP + lx + 1] = D[(byl + 1) * WP + lx + 1];
    };
    if (rx_ || ry_) {
      recopy(Dold);
      __syncthreads();
    }
#pragma unroll
    for (int k = 1; k <= NU; ++k) {
#pragma unroll
      for (int s = 0; s < NS; ++s) at(Dnew, cb[s]) = (sreg[s] + ax * at(Dold, ofx[s]) + ay * at(Dold, ofy[s])) * ireg[s];
      __syncthreads();
      if (rx_ || ry_) {
        recopy(Dnew);
        __syncthreads();
      }
      C* t = Dold;
      Dold = Dnew;
      Dnew = t;
    }
    // store the tile: column tx, rows ty + RSTEP k (pofs and pmask give the
    // global offset of row 0 and the rows inside the domain; the region's
    // cell of row 0 moves by a constant RSTEP WP per row block)
    const unsigned db = (unsigned)((ty + (syp ? NU : 0) + 1) * WP + tx + (sxp ? NU : 0) + 1) * sizeof(C);
    const size_t nbase = (size_t)n * npix + pofs;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (!((pmask >> k) & 1)) continue;
      const C d = at(Dold, db + (unsigned)(RSTEP * k * WP * sizeof(C)));
      const size_t gi = nbase + (size_t)(RSTEP * k) * nx;
      if (MODE == UP_CORR) {
        a.delta_out[gi] = d;
      } else {
        const C pn = pin[k] + d;
        Conv<T>::st(a.psi_out + gi, pn);
        phi_acc[k] += dr.w * stored<T, C>(pn);
      }
    }
    if (!(NU & 1)) {  // the buffer without this direction's result starts the next one
      Dinit = Dnew;
      Dother = Dold;
    }
  }
  if (MODE == UP_UPDATE) {
    C* ph = a.phi_part + (size_t)chunk * npix;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int gx = x0 + tx, gy = y0 + ty + RSTEP * k;
      if (gx < nx && gy < ny) ph[(size_t)gy * nx + gx] = phi_acc[k];
    }
  }
}

template <typename T, typename C, int MODE, int NU>
__global__ void __launch_bounds__(UNT, 3) k_upwind(const UpArgs<T, C> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  pdl_launch();
  upwind_tile<T, C, MODE, NU, UT>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// Finest-level upwind Jacobi with the update (UP_UPDATE) in streaming form,
// FP32 compute, psi stored in FP32, BF16 or FP16: no barriers after the set-up.  A warp owns 64 consecutive columns
// (two per lane) and walks a band of USR rows in the sweep order of the
// direction, all nu sweep levels at once: level k of a node needs level k-1
// of its x-upstream neighbour (the lane's other column, or the adjacent
// lane's by shuffle) and of its y-upstream neighbour (the previous row, kept
// in registers).  The UH columns on the x-upwind side (4 for FP32 storage, 8
// for BF16/FP16, nu <= 4: every window starts on a 16-byte boundary, as TMA
// needs) and the nu rows before the band are halo: a value there is exact
// only up to the level of its distance from the window's upwind edge, so the
// 64 - UH downwind columns and the band's rows are exact after nu levels.
// Each warp stages by TMA, into two buffers of its own with one mbarrier
// each, the source over the nu + USR rows, psi over the band and the rows of
// the coarser correction (UpSamp parents, x coarsened by 2), and sigma_t
// once over the union of the windows of both sign combinations; the next
// direction's copies are issued before the warp waits on the current one,
// so they land while it sweeps.  The chunk's direction table sits in shared
// memory.  Out-of-domain nodes (zero-filled by the copies) get inverse
// diagonal 0 and stay 0: the vacuum halo; on a reflective incoming side the
// boundary node reads its own previous level (the halo copy of the tiled
// kernel).  The update psi += delta and the scalar-flux partial sums over
// the chunk's directions are fused into the band's rows.
constexpr int USR = 8;       // output rows per warp band
constexpr int US_WARPS = 4;  // warps per CTA
constexpr int US_W = 64;     // columns of a warp's window
template <typename T> constexpr int us_uh() { return sizeof(T) == 2 ? 8 : 4; }  // halo columns
constexpr int US_CW = US_W / 2 + 4;  // coarse window columns (x coarsened by 2, start rounded down to 4)
constexpr int US_DMAX = 64;  // directions per chunk (at most 64 chunks of the direction count)
// staging per warp (floats, each part 128-byte aligned): sigma_t over
// [USR + 2 nu][64 + UH], then two buffers of source [ROWS][64], psi
// [USR][64] (storage type) and coarse correction [ROWS][US_CW]
template <typename T, int NU> struct UsBuf {
  static constexpr int ROWS = USR + NU, UH = us_uh<T>();
  static constexpr int rnd(int v) { return (v + 31) / 32 * 32; }
  static constexpr int SIGW = US_W + UH, SIGH = USR + 2 * NU;
  static constexpr int SIG = 0, B0 = rnd(SIGH * SIGW);
  static constexpr int SRC = 0, PSI = rnd(ROWS * US_W), CRS = PSI + rnd(USR * US_W * (int)sizeof(T) / 4);
  static constexpr int BUF = CRS + rnd(ROWS * US_CW), WARP = B0 + 2 * BUF;
};
template <typename T> __device__ __forceinline__ float2 ld_pair(const T* p) {
  if constexpr (sizeof(T) == 4) return *reinterpret_cast<const float2*>(p);
  else return make_float2(Conv<T>::ld(p), Conv<T>::ld(p + 1));
}
template <typename T> __device__ __forceinline__ void st_pair(T* p, float2 v) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = v;
  } else {
    T t[2];
    Conv<T>::st(&t[0], v.x);
    Conv<T>::st(&t[1], v.y);
    *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<const uint32_t*>(t);
  }
}
struct UsMaps {
  CUtensorMap src, sig, psi, crs;
};

template <typename T, int NU, bool SXP, bool SYP>
__device__ __forceinline__ void upstream_tile(const UpArgs<T, float>& a, const Dir<float>& dr, int n, int xw,
                                              int yb, int lane, const float* sigw, const float* buf, int cx0,
                                              int cy0, float2 (&phi)[USR]) {
  constexpr int ROWS = USR + NU, UH = us_uh<T>();
  using B = UsBuf<T, NU>;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;
  const int x0 = xw - (SXP ? UH : 0), r0 = SYP ? yb - NU : yb;  // window origin
  const int c0 = x0 + 2 * lane;                                     // this lane's columns c0, c0 + 1
  const bool cin = c0 >= 0 && c0 < nx;                              // nx even: both or neither
  T* pout = a.psi_out + (size_t)n * npix;
  const int shy = a.fy >> 1;
  const bool rx = SXP ? (a.bc.xlo == BC_REFLECTIVE && c0 == 0) : (a.bc.xhi == BC_REFLECTIVE && c0 + 1 == nx - 1);
  const int ybnd = SYP ? 0 : ny - 1;
  const bool ry = SYP ? a.bc.ylo == BC_REFLECTIVE : a.bc.yhi == BC_REFLECTIVE;
  const bool outl = SXP ? 2 * lane >= UH : 2 * lane < US_W - UH;
  const bool crs = a.init_mode == INIT_UPSAMPLE;
  const int cxl = (c0 >> 1) - cx0;                         // both columns' coarse column
  const int sgc = c0 - (xw - UH);                          // column in the sigma window
  const float2 ax = make_float2(dr.ax, dr.ax), ay = make_float2(dr.ay, dr.ay);
  const float axy = dr.ax + dr.ay;
  float2 prev[NU];
#pragma unroll
  for (int k = 0; k < NU; ++k) prev[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int it = 0; it < ROWS; ++it) {
    const int y = SYP ? yb - NU + it : yb + USR - 1 + NU - it;
    const int ri = y - r0;  // row in the staged window
    const bool in = cin && y >= 0 && y < ny;
    const float2 src = *reinterpret_cast<const float2*>(buf + B::SRC + ri * US_W + 2 * lane);
    const float2 sg = *reinterpret_cast<const float2*>(sigw + (y - (yb - NU)) * B::SIGW + sgc);
    float2 d = make_float2(0.f, 0.f);
    if (crs) d.x = d.y = buf[B::CRS + ((y >> shy) - cy0) * US_CW + cxl];
    const float2 inv = in ? make_float2(rcp_(axy + sg.x), rcp_(axy + sg.y)) : make_float2(0.f, 0.f);
    const bool ryb = ry && y == ybnd;
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      float2 ux;
      if (SXP) {
        ux.x = __shfl_up_sync(0xffffffffu, d.y, 1);
        if (rx) ux.x = d.x;
        ux.y = d.x;
      } else {
        ux.x = d.y;
        ux.y = __shfl_down_sync(0xffffffffu, d.x, 1);
        if (rx) ux.y = d.y;
      }
      const float2 uy = ryb ? d : prev[k];
      prev[k] = d;
      d = __fmul2_rn(__ffma2_rn(ax, ux, __ffma2_rn(ay, uy, src)), inv);  // the shuffle's value last
    }
    if (it >= NU) {
      const int orow = SYP ? it - NU : USR - 1 + NU - it;
      float2 pv = make_float2(0.f, 0.f);
      if (in && outl) {
        const float2 p = ld_pair(reinterpret_cast<const T*>(buf + B::PSI) + orow * US_W + 2 * lane);
        const float2 pn = make_float2(p.x + d.x, p.y + d.y);
        st_pair(pout + (size_t)y * nx + c0, pn);
        pv = make_float2(dr.w * stored<T, float>(pn.x), dr.w * stored<T, float>(pn.y));
      }
      if (SXP) {  // lane j: columns xw + 2j, xw + 2j + 1
        pv.x = __shfl_down_sync(0xffffffffu, pv.x, UH / 2);
        pv.y = __shfl_down_sync(0xffffffffu, pv.y, UH / 2);
      }
      phi[orow].x += pv.x;
      phi[orow].y += pv.y;
    }
  }
}

template <typename T, int NU>
__global__ void __launch_bounds__(US_WARPS * 32, 3) k_upwind_stream(const UpArgs<T, float> a, int ncg, int nbands,
                                                                    const __grid_constant__ UsMaps maps) {
  constexpr int UH = us_uh<T>(), OUTW = US_W - UH, ROWS = USR + NU;
  using B = UsBuf<T, NU>;
  extern __shared__ __align__(128) unsigned char us_smem[];
  __shared__ Dir<float> sdir[US_DMAX];
  __shared__ int spar[US_DMAX];
  pdl_wait();
  pdl_launch();
  __shared__ __align__(8) uint64_t sbar[US_WARPS][3];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int chunk = blockIdx.y;
  const int n_begin = chunk * a.dpc, n_end = min((chunk + 1) * a.dpc, a.nd);
  const bool crs = a.init_mode == INIT_UPSAMPLE;
  for (int i = threadIdx.x; i < n_end - n_begin; i += blockDim.x) {
    sdir[i] = a.dir[n_begin + i];
    spar[i] = crs ? a.parent[n_begin + i] : 0;
  }
  __syncthreads();
  const int wid = blockIdx.x * US_WARPS + wl;
  if (wid >= ncg * nbands) return;  // whole warps only: no barrier below
  const int xw = (wid % ncg) * OUTW, yb = (wid / ncg) * USR;
  float* wbase = reinterpret_cast<float*>(us_smem) + (size_t)wl * B::WARP;
  const float* sigw = wbase + B::SIG;
  float* bufs = wbase + B::B0;
  uint64_t* bar = sbar[wl];
  const int shy = a.fy >> 1;
  const uint32_t bytes =
      (uint32_t)(ROWS * US_W * sizeof(float) + USR * US_W * sizeof(T) + (crs ? ROWS * US_CW * sizeof(float) : 0));
  auto issue = [&](int i, int b) {  // lane 0: direction n_begin + i into buffer b
    const Dir<float>& dr = sdir[i];
    const int x0 = xw - (dr.mu > 0.f ? UH : 0), r0 = dr.nu > 0.f ? yb - NU : yb;
    float* dst = bufs + b * B::BUF;
    mbar_expect_tx(&bar[b], bytes);
    tma_load_3d(dst + B::SRC, &maps.src, &bar[b], x0, r0, n_begin + i);
    tma_load_3d(dst + B::PSI, &maps.psi, &bar[b], x0, yb, n_begin + i);
    if (crs) tma_load_3d(dst + B::CRS, &maps.crs, &bar[b], (x0 >> 1) & ~3, r0 >> shy, spar[i]);
  };
  if (lane == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(&bar[b], 1);
    mbar_fence_init();
    mbar_expect_tx(&bar[2], (uint32_t)(B::SIGH * B::SIGW * sizeof(float)));
    tma_load_3d(wbase + B::SIG, &maps.sig, &bar[2], xw - UH, yb - NU, 0);
    if (n_begin < n_end) issue(0, 0);
  }
  __syncwarp();
  bool ok = mbar_wait_bounded(&bar[2], 0);
  float2 phi[USR];
#pragma unroll
  for (int k = 0; k < USR; ++k) phi[k] = make_float2(0.f, 0.f);
  uint32_t parity = 0;  // bit b: parity of buffer b's next completion
  for (int i = 0; ok && i < n_end - n_begin; ++i) {
    const int b = i & 1;
    __syncwarp();  // every lane is done with the other buffer (the previous direction)
    if (lane == 0 && i + 1 < n_end - n_begin) {
      fence_proxy_async();
      issue(i + 1, b ^ 1);
    }
    ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[b], (parity >> b) & 1u));
    parity ^= 1u << b;
    if (!ok) {  // copy engine stalled: drain the other copy, then flag and leave
      if (lane == 0 && i + 1 < n_end - n_begin) mbar_wait_bounded(&bar[b ^ 1], (parity >> (b ^ 1)) & 1u);
      break;
    }
    const Dir<float> dr = sdir[i];
    const int n = n_begin + i;
    const int x0 = xw - (dr.mu > 0.f ? UH : 0), r0 = dr.nu > 0.f ? yb - NU : yb;
    const int cx0 = (x0 >> 1) & ~3, cy0 = r0 >> shy;
    const float* buf = bufs + b * B::BUF;
    const bool sxp = dr.mu > 0.f, syp = dr.nu > 0.f;
    if (sxp && syp) upstream_tile<T, NU, true, true>(a, dr, n, xw, yb, lane, sigw, buf, cx0, cy0, phi);
    else if (sxp) upstream_tile<T, NU, true, false>(a, dr, n, xw, yb, lane, sigw, buf, cx0, cy0, phi);
    else if (syp) upstream_tile<T, NU, false, true>(a, dr, n, xw, yb, lane, sigw, buf, cx0, cy0, phi);
    else upstream_tile<T, NU, false, false>(a, dr, n, xw, yb, lane, sigw, buf, cx0, cy0, phi);
  }
  if (!ok) {
    if (lane == 0) atomicExch(a.err, 1);
    return;
  }
  const int col = xw + 2 * lane;
  if (2 * lane < OUTW && col < a.nx) {
    float* ph = a.phi_part + (size_t)chunk * a.nx * a.ny;
#pragma unroll
    for (int k = 0; k < USR; ++k)
      if (yb + k < a.ny) *reinterpret_cast<float2*>(ph + (size_t)(yb + k) * a.nx + col) = phi[k];
  }
}

// Coarse cells [id0, id1) of the restriction fine -> coarse (Sec. 2.5),
// strided over the CTA's threads starting at `first` with step `stride`.
template <typename C>
__device__ __forceinline__ void restrict_cells(const C* __restrict__ fine, C* __restrict__ coarse,
                                               const C* __restrict__ rcoef, int nx, int ny, int nr, int nc, int nxc,
                                               int nyc, int nrc, int ncc, int fx, int fy, int fr, int fc,
                                               size_t first, size_t stride, size_t id1) {
  for (size_t id = first; id < id1; id += stride) {
    const int X = id % nxc;
    const int Y = (id / nxc) % nyc;
    const int N = id / ((size_t)nxc * nyc);
    const int f = N / (nrc * ncc), J = (N % (nrc * ncc)) / ncc, I = N % ncc;
    C acc = C(0);
    for (int aa = 0; aa < fr; ++aa) {
      const int j = J * fr + aa;
      if (j >= nr) continue;
      for (int bb = 0; bb < fc; ++bb) {
        const int i = I * fc + bb;
        if (i >= nc) continue;
        const int n = f * nr * nc + j * nc + i;
        const C w = rcoef[n];
        for (int yy = 0; yy < fy; ++yy) {
          const int y = Y * fy + yy;
          if (y >= ny) continue;
          for (int xx = 0; xx < fx; ++xx) {
            const int x = X * fx + xx;
            if (x >= nx) continue;
            acc += w * fine[((size_t)n * ny + y) * nx + x];
          }
        }
      }
    }
    coarse[id] = acc;
  }
}

// Persistent batched coarse correction: each CTA takes (segment, block)
// tasks from a global counter until the queue is empty; before a task, its
// thread 0 waits (bounded, about a second) until the previous segment of the
// same problem has all its blocks finished, and after the task it publishes
// the block (fence, then counter).  The queue lists every prerequisite
// before its dependents, so the tasks a CTA waits on were taken earlier by
// running CTAs: no deadlock whatever the grid.  A wait that gives up sets
// the error word and ends the CTA.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
template <int NU, int TU>
__global__ void __launch_bounds__(UNT) k_coarse_batch(const CoarseBatch cb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task, s_ok;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = (int)atomicAdd(cb.head, 1u);
      int ok = 1;
      if (t < cb.ntasks) {
        const int prev = cb.seg[cb.task[t].x].prev;
        if (prev >= 0) {
          const unsigned need = (unsigned)cb.seg[prev].blocks;
          for (int it = 0; ld_acquire(cb.done + prev) < need; ++it) {
            if (it >= (1 << 22)) {
              ok = 0;
              break;
            }
            __nanosleep(256);
          }
        }
      }
      s_task = t;
      s_ok = ok;
    }
    __syncthreads();
    const int t = s_task;
    if (t >= cb.ntasks) return;
    if (!s_ok) {
      if (threadIdx.x == 0) atomicExch(cb.err, 1);
      return;
    }
    const int2 tk = cb.task[t];
    const CoarseSeg sg = cb.seg[tk.x];
    if (sg.type == 0) {
      const CoarseRestrict& r = cb.ra[sg.arg];
      const size_t total = (size_t)8 * r.nrc * r.ncc * r.nyc * r.nxc;
      const size_t id0 = (size_t)tk.y * kCoarseCells, id1 = min(total, id0 + (size_t)kCoarseCells);
      restrict_cells<float>(r.fine, r.coarse, r.rcoef, r.nx, r.ny, r.nr, r.nc, r.nxc, r.nyc, r.nrc, r.ncc, r.fx, r.fy,
                            r.fr, r.fc, id0 + threadIdx.x, blockDim.x, id1);
    } else {
      upwind_tile<float, float, UP_CORR, NU, TU>(cb.ua[sg.arg], tk.y % sg.tiles, tk.y / sg.tiles, smem_raw);
    }
    __syncthreads();  // the block's writes precede its publication
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(cb.done + tk.x, 1u);
    }
  }
}

template <typename C>
__global__ void k_restrict(const C* __restrict__ fine, C* __restrict__ coarse, const C* __restrict__ rcoef,
                           int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc, int ncc, int fx, int fy,
                           int fr, int fc) {
  pdl_wait();
  pdl_launch();
  const size_t total = (size_t)8 * nrc * ncc * nyc * nxc;
  restrict_cells<C>(fine, coarse, rcoef, nx, ny, nr, nc, nxc, nyc, nrc, ncc, fx, fy, fr, fc,
                    blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x, total);
}

// The restriction of a level whose coarse cells all have their 2 x 2 node
// and 2 x 2 direction children, with coarse rows of a multiple of 4 nodes:
// thread (q, Y, N) forms coarse nodes 4q .. 4q+3 of coarse row Y and
// direction N from 16-byte row loads, each cell summed in restrict_cells'
// order (children (j, i), then fine rows, then fine columns), so the two
// kernels agree bit for bit.
__global__ void k_restrict4(const float* __restrict__ fine, float* __restrict__ coarse,
                            const float* __restrict__ rcoef, int nx, int ny, int nr, int nc, int nxc, int nyc,
                            int nrc, int ncc) {
  pdl_wait();
  pdl_launch();
  const int q = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y * blockDim.y + threadIdx.y, N = blockIdx.z;
  if (4 * q >= nxc || Y >= nyc) return;
  const int f = N / (nrc * ncc), J = (N % (nrc * ncc)) / ncc, I = N % ncc;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int aa = 0; aa < 2; ++aa)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int n = f * nr * nc + (2 * J + aa) * nc + 2 * I + bb;
      const float w = rcoef[n];
#pragma unroll
      for (int yy = 0; yy < 2; ++yy) {
        const float* row = fine + ((size_t)n * ny + 2 * Y + yy) * nx + 8 * q;
        const float4 u = *reinterpret_cast<const float4*>(row), v = *reinterpret_cast<const float4*>(row + 4);
        const float x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc[k] += w * x[2 * k];
          acc[k] += w * x[2 * k + 1];
        }
      }
    }
  *reinterpret_cast<float4*>(coarse + ((size_t)N * nyc + Y) * nxc + 4 * q) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// k_restrict4 for a fine residual assembled here: r = r' + b, with r' the
// residual of a launch with zero source (-A psi) and b isotropic; r is
// written back in place (b - A psi with one rounding, as the residual kernel
// forms it), restricted exactly as k_restrict4 restricts r, and the CTA's
// share of the weighted squared norm sum p_n dx dy r^2 written to
// part[block] (the fine nodes of the CTA's coarse cells).
__global__ void __launch_bounds__(256) k_restrict4_rb(float* __restrict__ r, const float* __restrict__ b,
                                                      float* __restrict__ coarse, const float* __restrict__ rcoef,
                                                      const Dir<float>* __restrict__ dir, double dxdy,
                                                      double* __restrict__ part, int nx, int ny, int nr, int nc,
                                                      int nxc, int nyc, int nrc, int ncc) {
  pdl_wait();
  pdl_launch();
  __shared__ double red[8];
  const int q = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y * blockDim.y + threadIdx.y, N = blockIdx.z;
  double nrm = 0.0;
  if (4 * q < nxc && Y < nyc) {
    const int f = N / (nrc * ncc), J = (N % (nrc * ncc)) / ncc, I = N % ncc;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int aa = 0; aa < 2; ++aa)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const int n = f * nr * nc + (2 * J + aa) * nc + 2 * I + bb;
        const float w = rcoef[n];
        float ns = 0.f;  // squares in FP32 (FP64 arithmetic is slow on this GPU), summed in FP64 below
#pragma unroll
        for (int yy = 0; yy < 2; ++yy) {
          float* row = r + ((size_t)n * ny + 2 * Y + yy) * nx + 8 * q;
          const float* brow = b + (size_t)(2 * Y + yy) * nx + 8 * q;
          const float4 u = *reinterpret_cast<const float4*>(row), v = *reinterpret_cast<const float4*>(row + 4);
          const float4 bu = *reinterpret_cast<const float4*>(brow), bv = *reinterpret_cast<const float4*>(brow + 4);
          const float x[8] = {bu.x + u.x, bu.y + u.y, bu.z + u.z, bu.w + u.w,
                              bv.x + v.x, bv.y + v.y, bv.z + v.z, bv.w + v.w};
          *reinterpret_cast<float4*>(row) = make_float4(x[0], x[1], x[2], x[3]);
          *reinterpret_cast<float4*>(row + 4) = make_float4(x[4], x[5], x[6], x[7]);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[k] += w * x[2 * k];
            acc[k] += w * x[2 * k + 1];
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) ns += x[k] * x[k];
        }
        nrm += (double)dir[n].w * (double)ns;
      }
    *reinterpret_cast<float4*>(coarse + ((size_t)N * nyc + Y) * nxc + 4 * q) =
        make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0) red[t >> 5] = nrm;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += red[w];
    part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum * dxdy;
  }
}

template <typename C>
__global__ void k_prolong(const C* __restrict__ coarse, C* __restrict__ fine, int nx, int ny, int nr, int nc,
                          int nxc, int nyc, int nrc, int ncc, int fx, int fy, int fr, int fc) {
  const size_t total = (size_t)8 * nr * nc * ny * nx;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int x = id % nx;
    const int y = (id / nx) % ny;
    const int n = id / ((size_t)nx * ny);
    const int f = n / (nr * nc), j = (n % (nr * nc)) / nc, i = n % nc;
    const int N = f * nrc * ncc + (j / fr) * ncc + i / fc;
    fine[id] = coarse[((size_t)N * nyc + y / fy) * nxc + x / fx];
  }
}

template <typename T, typename C>
__global__ void k_phi_partial(const T* __restrict__ psi, C* __restrict__ part, const Dir<C>* __restrict__ dir,
                              int npix, int nd, int dpc, int nchunk) {
  pdl_wait();
  pdl_launch();
  const size_t total = (size_t)nchunk * npix;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
    const int pix = id % npix;
    const int c = id / npix;
    C acc = C(0);
    const int n1 = min((c + 1) * dpc, nd);
    for (int n = c * dpc; n < n1; ++n) acc += dir[n].w * Conv<T>::ld(psi + (size_t)n * npix + pix);
    part[id] = acc;
  }
}

template <typename C>
__global__ void k_source(const C* __restrict__ src_g, const C* __restrict__ sigs_g, const C* __restrict__ phi_part,
                         int G, int g, int nchunk, int npix, C* __restrict__ b, C* __restrict__ qfix,
                         double* __restrict__ qn2_part) {
  pdl_wait();
  pdl_launch();
  __shared__ double red[8];
  double acc = 0.0;
  const C inv4pi = C(0.07957747154594767);  // 1 / (4 pi)
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < npix; pix += gridDim.x * blockDim.x) {
    C q = src_g[pix], self = C(0);
    for (int h = 0; h < G; ++h) {
      const C sg = sigs_g[(size_t)h * npix + pix];
      C phi = C(0);
      for (int c = 0; c < nchunk; ++c) phi += phi_part[((size_t)h * nchunk + c) * npix + pix];
      if (h == g) self = sg * phi * inv4pi;
      else q += sg * phi * inv4pi;
    }
    b[pix] = q + self;
    if (qfix) qfix[pix] = q;
    acc += (double)q * (double)q;
  }
  if (!qn2_part) return;  // no norm wanted (uniform over the grid)
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    qn2_part[blockIdx.x] = s;
  }
}

template <typename C>
__global__ void k_phi_sum(const C* __restrict__ part, int nchunk, int npix, C* __restrict__ phi) {
  pdl_wait();
  pdl_launch();
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < npix; pix += gridDim.x * blockDim.x) {
    C acc = C(0);
    for (int c = 0; c < nchunk; ++c) acc += part[(size_t)c * npix + pix];
    phi[pix] = acc;
  }
}

// one block: the deterministic sum of part[0..n) into out[0]
__device__ __forceinline__ void block_sum(const double* __restrict__ part, int n, double* __restrict__ out,
                                          double* red) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[0] = s;
  }
}

__global__ void k_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  pdl_wait();
  pdl_launch();
  __shared__ double red[32];
  block_sum(part, n, out, red);
}

__global__ void k_sum2(const double* __restrict__ part_a, int na, double* __restrict__ out_a,
                       const double* __restrict__ part_b, int nb, double* __restrict__ out_b) {
  pdl_wait();
  pdl_launch();
  __shared__ double red[2][32];
  block_sum(part_a, na, out_a, red[0]);
  block_sum(part_b, nb, out_b, red[1]);
}

// one-block deterministic sum (the same reduction as launch_sum, local to each TU)
__global__ void k_sum_local(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[0] = s;
  }
}
inline void k_sum_fwd(const double* part, int n, double* out, cudaStream_t s) { k_sum_local<<<1, 1024, 0, s>>>(part, n, out); }

inline int grid_for(size_t total, int threads) {
  size_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}

template <typename T, typename C, int MODE, int NU>
cudaError_t launch_up_nu(const UpArgs<T, C>& a, int nchunk, cudaStream_t s) {
  constexpr int WP = UT + NU + 2, WS = UT + 2 * NU;
  const size_t smem = (2 * ((size_t)WP * WP + 1) + (size_t)WS * WS) * sizeof(C);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_upwind<T, C, MODE, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tiles_y = (a.ny + UT - 1) / UT;
  dim3 grid(a.tiles_x * tiles_y, nchunk);
  return launch_pdl(k_upwind<T, C, MODE, NU>, grid, dim3(UNT), smem, s, a);
}

template <typename T, typename C, int MODE>
cudaError_t launch_up_mode(const UpArgs<T, C>& a, int nchunk, cudaStream_t s) {
  switch (a.nu) {
    case 1: return launch_up_nu<T, C, MODE, 1>(a, nchunk, s);
    case 2: return launch_up_nu<T, C, MODE, 2>(a, nchunk, s);
    case 3: return launch_up_nu<T, C, MODE, 3>(a, nchunk, s);
    case 4: return launch_up_nu<T, C, MODE, 4>(a, nchunk, s);
    case 5: return launch_up_nu<T, C, MODE, 5>(a, nchunk, s);
    case 6: return launch_up_nu<T, C, MODE, 6>(a, nchunk, s);
    case 7: return launch_up_nu<T, C, MODE, 7>(a, nchunk, s);
    case 8: return launch_up_nu<T, C, MODE, 8>(a, nchunk, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int NU>
cudaError_t launch_up_stream(const UpArgs<T, float>& a, const UsMaps& maps, int nchunk, cudaStream_t s) {
  constexpr int OUTW = US_W - us_uh<T>();
  constexpr size_t smem = (size_t)US_WARPS * UsBuf<T, NU>::WARP * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(k_upwind_stream<T, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int ncg = (a.nx + OUTW - 1) / OUTW, nbands = (a.ny + USR - 1) / USR;
  const int warps = ncg * nbands;
  dim3 grid((warps + US_WARPS - 1) / US_WARPS, nchunk);
  return launch_pdl(k_upwind_stream<T, NU>, grid, dim3(US_WARPS * 32), smem, s, a, ncg, nbands, maps);
}

// Tensor maps of the streaming kernel's windows, or false when the layout
// does not allow them (rows not 16-byte multiples, unaligned bases, x not
// coarsened by 2, more than US_DMAX directions per chunk).
template <typename T> bool up_stream_maps(const UpArgs<T, float>& a, UsMaps* m) {
  const int rows = USR + a.nu, uh = us_uh<T>();
  if (a.src_stride != (size_t)a.nx * a.ny || !a.err || a.dpc > US_DMAX || a.nx % 4) return false;
  const CUtensorMapDataType pt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (!encode_tmap_3d(&m->src, a.src, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.nx, a.ny, a.nd, US_W, rows)) return false;
  if (!encode_tmap_3d(&m->sig, a.sig, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.nx, a.ny, 1, US_W + uh, USR + 2 * a.nu))
    return false;
  if (!encode_tmap_3d(&m->psi, a.psi_in, pt, sizeof(T), a.nx, a.ny, a.nd, US_W, USR)) return false;
  if (a.init_mode == INIT_UPSAMPLE) {
    if (a.fx != 2) return false;
    const int ndc = 8 * a.nrc * a.ncc;
    if (!encode_tmap_3d(&m->crs, a.init, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.nxc, a.nyc, ndc, US_CW, rows))
      return false;
  } else if (a.init_mode != INIT_ZERO) {
    return false;
  }
  return true;
}

}  // namespace

// The finest level's sweeps with the update run in the streaming kernel
// (FP32 compute, rows of 16-byte multiples, 16-byte aligned buffers);
// the correction levels and other layouts in the tiled one.
template <typename T, typename C>
cudaError_t launch_upwind(const UpArgs<T, C>& a, int mode, int nchunk, cudaStream_t s) {
  if constexpr (std::is_same<C, float>::value) {
    UsMaps maps;
    memset(&maps, 0, sizeof(maps));
    if (mode == UP_UPDATE && a.nu <= 4 && up_stream_maps<T>(a, &maps)) {
      switch (a.nu) {
        case 1: return launch_up_stream<T, 1>(a, maps, nchunk, s);
        case 2: return launch_up_stream<T, 2>(a, maps, nchunk, s);
        case 3: return launch_up_stream<T, 3>(a, maps, nchunk, s);
        case 4: return launch_up_stream<T, 4>(a, maps, nchunk, s);
      }
    }
  }
  return mode == UP_CORR ? launch_up_mode<T, C, UP_CORR>(a, nchunk, s) : launch_up_mode<T, C, UP_UPDATE>(a, nchunk, s);
}

template <typename C>
cudaError_t launch_restrict(const C* fine, C* coarse, const C* rcoef, int nx, int ny, int nr, int nc, int nxc,
                            int nyc, int nrc, int ncc, int fx, int fy, int fr, int fc, cudaStream_t s) {
  const size_t total = (size_t)8 * nrc * ncc * nyc * nxc;
  if constexpr (std::is_same<C, float>::value) {
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) % 16) == 0; };
    if (fx == 2 && fy == 2 && fr == 2 && fc == 2 && nx == 2 * nxc && ny == 2 * nyc && nr == 2 * nrc &&
        nc == 2 * ncc && nxc % 4 == 0 && nyc <= 65535 * 8 && 8 * nrc * ncc <= 65535 && al(fine) && al(coarse)) {
      const dim3 block(32, 8), grid((nxc / 4 + 31) / 32, (nyc + 7) / 8, 8 * nrc * ncc);
      return launch_pdl(k_restrict4, grid, block, 0, s, fine, coarse, rcoef, nx, ny, nr, nc, nxc, nyc, nrc, ncc);
    }
  }
  return launch_pdl(k_restrict<C>, dim3(grid_for(total, 256)), dim3(256), 0, s, fine, coarse, rcoef, nx, ny, nr, nc,
                    nxc, nyc, nrc, ncc, fx, fy, fr, fc);
}

template <typename C>
cudaError_t launch_prolong(const C* coarse, C* fine, int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc,
                           int ncc, int fx, int fy, int fr, int fc, cudaStream_t s) {
  const size_t total = (size_t)8 * nr * nc * ny * nx;
  k_prolong<C><<<grid_for(total, 256), 256, 0, s>>>(coarse, fine, nx, ny, nr, nc, nxc, nyc, nrc, ncc, fx, fy, fr,
                                                     fc);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t launch_phi_partial(const T* psi, C* part, const Dir<C>* dir, int nx, int ny, int nd, int dpc,
                               int nchunk, cudaStream_t s) {
  const int npix = nx * ny;
  return launch_pdl(k_phi_partial<T, C>, dim3(grid_for((size_t)nchunk * npix, 256)), dim3(256), 0, s, psi, part, dir,
                    npix, nd, dpc, nchunk);
}

template <typename C>
cudaError_t launch_source(const C* src_g, const C* sigs_g, const C* phi_part, int G, int g, int nchunk, int npix,
                          C* b, C* qfix, double* qn2_part, int nblocks, cudaStream_t s) {
  return launch_pdl(k_source<C>, dim3(nblocks), dim3(256), 0, s, src_g, sigs_g, phi_part, G, g, nchunk, npix, b, qfix,
                    qn2_part);
}

template <typename C>
cudaError_t launch_phi_sum(const C* part, int nchunk, int npix, C* phi, cudaStream_t s) {
  return launch_pdl(k_phi_sum<C>, dim3(grid_for(npix, 256)), dim3(256), 0, s, part, nchunk, npix, phi);
}

namespace {
// sum over the grid of (phi - phi_prev)^2 (per-block partials), phi = sum of chunks
template <typename C>
__global__ void k_dphi_norm(const C* __restrict__ phi_part, int nchunk, const C* __restrict__ phi_prev, int npix,
                            double* __restrict__ part) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    C v = C(0);
    for (int c = 0; c < nchunk; ++c) v += phi_part[(size_t)c * npix + p];
    const double d = (double)v - (double)phi_prev[p];
    acc += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}
// Features of the learned correction on the coarse canvas W8 x H8: canvas
// pixel (X, Y) averages the fine nodes [X f, X f + f) x [Y f, Y f + f) of
// the grid (cut at its edge; zeros outside the ncx x ncy covered pixels):
//   0 mean rho (normalised afterwards),  1 log(mean sigma_t * f dx + 1e-3) / 4,
//   2 mean sigma_s / mean sigma_t,       3 mean (phi - phi_prev) (normalised
//   afterwards; 0 without phi_prev).
// part[blk], part[nblk + blk]: partial sums of channel 0 and 3 squared.
template <typename C>
__global__ void k_learn_coarse(const C* __restrict__ rho_part, const C* __restrict__ phi_part,
                               const C* __restrict__ phi_prev, int nchunk, const C* __restrict__ sigt,
                               const C* __restrict__ sigs_gg, int nx, int ny, int f, int ncx, int ncy, int W8, int H8,
                               double dXc, float* __restrict__ feat, double* __restrict__ part) {
  __shared__ double red0[8], red3[8];
  const size_t npix = (size_t)nx * ny;
  double a0 = 0.0, a3 = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < W8 * H8; q += gridDim.x * blockDim.x) {
    const int X = q % W8, Y = q / W8;
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
    if (X < ncx && Y < ncy) {
      double r = 0.0, st = 0.0, ss = 0.0, dp = 0.0;
      int cnt = 0;
      for (int y = Y * f; y < min(Y * f + f, ny); ++y)
        for (int x = X * f; x < min(X * f + f, nx); ++x) {
          const size_t p = (size_t)y * nx + x;
          C v = C(0);
          for (int c = 0; c < nchunk; ++c) v += rho_part[(size_t)c * npix + p];
          r += (double)v;
          st += (double)sigt[p];
          ss += (double)sigs_gg[p];
          if (phi_prev) {
            C ph = C(0);
            for (int c = 0; c < nchunk; ++c) ph += phi_part[(size_t)c * npix + p];
            dp += (double)ph - (double)phi_prev[p];
          }
          ++cnt;
        }
      const double inv = 1.0 / (double)cnt;
      f0 = (float)(r * inv);
      f1 = (float)(0.25 * log(st * inv * dXc + 1e-3));
      f2 = st > 0 ? (float)(ss / st) : 0.f;
      f3 = (float)(dp * inv);
      a0 += (double)f0 * f0;
      a3 += (double)f3 * f3;
    }
    float* o = feat + (size_t)q * kLearnFeatures;
    o[0] = f0;
    o[1] = f1;
    o[2] = f2;
    o[3] = f3;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a3 += __shfl_xor_sync(0xffffffffu, a3, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red0[threadIdx.x >> 5] = a0;
    red3[threadIdx.x >> 5] = a3;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s3 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red0[w];
      s3 += red3[w];
    }
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s3;
  }
}
// channels 0 and 3 divided by their rms over the covered canvas pixels;
// scale_out = rms of channel 0
__global__ void k_learn_normalise(float* __restrict__ feat, int n, int ncov, const double* __restrict__ d_sum,
                                  float* __restrict__ scale_out) {
  const double r0 = sqrt(d_sum[0] / (double)ncov), r3 = sqrt(d_sum[1] / (double)ncov);
  const float i0 = r0 > 0 ? (float)(1.0 / r0) : 0.f, i3 = r3 > 0 ? (float)(1.0 / r3) : 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) scale_out[0] = (float)r0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    feat[(size_t)q * kLearnFeatures + 0] *= i0;
    feat[(size_t)q * kLearnFeatures + 3] *= i3;
  }
}
// Learned correction as a P1 angular flux (Sec. 2.5 scalar flux, Fick's law
// closure): e = the U-net output on the coarse canvas, interpolated
// bilinearly to the fine nodes (canvas pixel X is centred on fine
// coordinate (X + 1/2) f - 1/2, clamped at the covered edge), becomes
// c_n = (e - (mu_n de/dx + nu_n de/dy) / sigma) / (4 pi), with
// sigma = max(sigma_t, 1 / domain length) and central differences
// (one-sided at the edges).  b_out = (sigma_s,gg / 4 pi) e is the in-group
// scattering source of c, so that a residual evaluation of c with b_out
// gives -L c.
template <typename T, typename C>
__global__ void k_learn_build(T* __restrict__ c_out, C* __restrict__ b_out, const float* __restrict__ delta,
                              const C* __restrict__ sigt, const C* __restrict__ sigs_gg,
                              const Dir<C>* __restrict__ dir, int nd, int nx, int ny, int W8, int f, int ncx, int ncy,
                              float inv_dx, float inv_dy, float inv_len) {
  const size_t npix = (size_t)nx * ny, total = (size_t)nd * npix;
  const float inv4pi = 0.07957747154594767f, invf = 1.f / (float)f;
  auto E = [&](int x, int y) {
    float u = ((float)x + 0.5f) * invf - 0.5f, v = ((float)y + 0.5f) * invf - 0.5f;
    u = fminf(fmaxf(u, 0.f), (float)(ncx - 1));
    v = fminf(fmaxf(v, 0.f), (float)(ncy - 1));
    const int i0 = (int)u, j0 = (int)v;
    const int i1 = min(i0 + 1, ncx - 1), j1 = min(j0 + 1, ncy - 1);
    const float tu = u - (float)i0, tv = v - (float)j0;
    const float a = delta[(size_t)j0 * W8 + i0], b = delta[(size_t)j0 * W8 + i1];
    const float c = delta[(size_t)j1 * W8 + i0], d = delta[(size_t)j1 * W8 + i1];
    return (1.f - tv) * ((1.f - tu) * a + tu * b) + tv * ((1.f - tu) * c + tu * d);
  };
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i % npix;
    const int n = (int)(i / npix);
    const int x = (int)(p % nx), y = (int)(p / nx);
    const float e = E(x, y);
    const int xl = x > 0 ? x - 1 : x, xr = x + 1 < nx ? x + 1 : x;
    const int yl = y > 0 ? y - 1 : y, yr = y + 1 < ny ? y + 1 : y;
    const float ex = xr > xl ? (E(xr, y) - E(xl, y)) * inv_dx / (float)(xr - xl) : 0.f;
    const float ey = yr > yl ? (E(x, yr) - E(x, yl)) * inv_dy / (float)(yr - yl) : 0.f;
    const float st = (float)sigt[p];
    const float sg = st > inv_len ? st : inv_len;
    const float v = (e - ((float)dir[n].mu * ex + (float)dir[n].nu * ey) / sg) * inv4pi;
    Conv<T>::st(c_out + i, (C)v);
    if (n == 0) b_out[p] = (C)((float)sigs_gg[p] * e * inv4pi);
  }
}
// partial sums of sum_n p_n dx dy r1 rc over one group (the residual weight)
template <typename C>
__global__ void k_learn_dot(const C* __restrict__ r1, const C* __restrict__ rc, const Dir<C>* __restrict__ dir,
                            size_t npix, int nd, double dxdy, double* __restrict__ part) {
  __shared__ double red[32];
  const size_t total = (size_t)nd * npix;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    acc += (double)dir[i / npix].w * (double)r1[i] * (double)rc[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s * dxdy;
  }
}
// Step length minimising the weighted residual norm along c:
// r(psi + alpha c) = r + alpha rc, alpha = -<r, rc> / <rc, rc>, then psi +=
// alpha c and the scalar-flux partials phi += alpha phi_c.
// ldot = {<r, rc>, <rc, rc>, sum phi_c^2, sum dphi^2} (dphi = the plain
// cycle's scalar-flux update); rn2 = <r, r>.  Guards: alpha = 0 when a sum is
// not finite, <rc, rc> = 0 or the predicted reduction of ||r||^2 is below
// 1e-4 (a step of rounding noise); |alpha| rms(phi_c) <= 1e3 rms(dphi) (any
// alpha between 0 and the minimiser still lowers the residual).  stat
// accumulates the residual reduction factor, the step count and the last
// alpha.
__device__ __forceinline__ double learn_alpha(const double* ldot, double rr) {
  const double d = ldot[0], nn = ldot[1], pc = ldot[2], dp = ldot[3];
  if (!(nn > 0.0) || !isfinite(nn) || !isfinite(d) || !isfinite(pc) || !isfinite(dp) || !(rr > 0.0)) return 0.0;
  if (d * d < 1e-4 * nn * rr) return 0.0;
  double al = -d / nn;
  const double cap = pc > 0.0 ? 1e3 * sqrt(dp / pc) : 0.0;
  return al > cap ? cap : (al < -cap ? -cap : al);
}
template <typename T, typename C>
__global__ void k_learn_update(T* __restrict__ psi, const T* __restrict__ c, size_t n, C* __restrict__ phi,
                               const C* __restrict__ phi_c, size_t nphi, const double* __restrict__ ldot,
                               const double* __restrict__ rn2, double* __restrict__ stat) {
  const double rr = rn2[0];
  const double al = learn_alpha(ldot, rr);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double after = rr + 2.0 * al * ldot[0] + al * al * ldot[1];
    stat[0] += (rr > 0.0 && after > 0.0) ? sqrt(after / rr) : 0.0;
    stat[1] += 1.0;
    stat[2] = al;
  }
  const C a = (C)al;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    Conv<T>::st(psi + i, (C)Conv<T>::ld(psi + i) + a * (C)Conv<T>::ld(c + i));
    if (i < nphi) phi[i] += a * phi_c[i];
  }
}
template <typename C>
__global__ void k_scale_to(const double* __restrict__ r64, C* __restrict__ out, double alpha, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (C)(alpha * r64[i]);
}
template <typename T>
__global__ void k_refine_update(double* __restrict__ psi64, const T* __restrict__ delta, double inv_alpha, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    psi64[i] += (double)Conv<T>::ld(delta + i) * inv_alpha;
}

}  // namespace

template <typename C>
cudaError_t launch_learn_features(const C* rho_part, int nchunk, const C* phi_part, const C* phi_prev, const C* sigt,
                                  const C* sigs_gg, double dx, int nx, int ny, int f, int W8, int H8, double* d_sum,
                                  double* d_part, float* feat, float* scale_out, cudaStream_t s) {
  const int ncx = (nx + f - 1) / f, ncy = (ny + f - 1) / f;
  k_learn_coarse<C><<<kLearnBlocks, 256, 0, s>>>(rho_part, phi_part, phi_prev, nchunk, sigt, sigs_gg, nx, ny, f, ncx,
                                                 ncy, W8, H8, dx * f, feat, d_part);
  k_sum_fwd(d_part, kLearnBlocks, d_sum, s);
  k_sum_fwd(d_part + kLearnBlocks, kLearnBlocks, d_sum + 1, s);
  k_learn_normalise<<<kLearnBlocks, 256, 0, s>>>(feat, W8 * H8, ncx * ncy, d_sum, scale_out);
  return cudaGetLastError();
}
template <typename T, typename C>
cudaError_t launch_learn_build(T* c_out, C* b_out, const float* delta, const C* sigt, const C* sigs_gg,
                               const Dir<C>* dir, int nd, int nx, int ny, int f, int W8, double dx, double dy,
                               double inv_len, cudaStream_t s) {
  const int ncx = (nx + f - 1) / f, ncy = (ny + f - 1) / f;
  k_learn_build<T, C><<<grid_for((size_t)nd * nx * ny, 256), 256, 0, s>>>(
      c_out, b_out, delta, sigt, sigs_gg, dir, nd, nx, ny, W8, f, ncx, ncy, (float)(1.0 / dx), (float)(1.0 / dy),
      (float)inv_len);
  return cudaGetLastError();
}
template <typename C>
cudaError_t launch_dphi_norm(const C* phi_part, int nchunk, const C* phi_prev, int npix, double* d_part, int nblk,
                             double* out, cudaStream_t s) {
  k_dphi_norm<C><<<nblk, 256, 0, s>>>(phi_part, nchunk, phi_prev, npix, d_part);
  k_sum_fwd(d_part, nblk, out, s);
  return cudaGetLastError();
}
template <typename C>
cudaError_t launch_learn_dot(const C* r1, const C* rc, const Dir<C>* dir, int nx, int ny, int nd, double dxdy,
                             double* part, int nblk, double* out, cudaStream_t s) {
  k_learn_dot<C><<<nblk, 256, 0, s>>>(r1, rc, dir, (size_t)nx * ny, nd, dxdy, part);
  k_sum_fwd(part, nblk, out, s);
  return cudaGetLastError();
}
template <typename T, typename C>
cudaError_t launch_learn_update(T* psi, const T* c, size_t n, C* phi, const C* phi_c, size_t nphi, const double* ldot,
                                const double* rn2, double* stat, cudaStream_t s) {
  k_learn_update<T, C><<<grid_for(n, 256), 256, 0, s>>>(psi, c, n, phi, phi_c, nphi, ldot, rn2, stat);
  return cudaGetLastError();
}
template <typename C>
cudaError_t launch_scale_to(const double* r64, C* out, double alpha, size_t n, cudaStream_t s) {
  k_scale_to<C><<<grid_for(n, 256), 256, 0, s>>>(r64, out, alpha, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_refine_update(double* psi64, const T* delta, double inv_alpha, size_t n, cudaStream_t s) {
  k_refine_update<T><<<grid_for(n, 256), 256, 0, s>>>(psi64, delta, inv_alpha, n);
  return cudaGetLastError();
}

#ifdef BTMG_MG_DEFINE_COMMON
namespace {
template <int NU, int TU>
cudaError_t launch_cb(const CoarseBatch& cb, int ctas, cudaStream_t s) {
  constexpr size_t smem = upwind_smem<float, NU, TU>();
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_coarse_batch<NU, TU><<<sms * ctas, UNT, smem, s>>>(cb);
  return cudaGetLastError();
}
}  // namespace
bool coarse_batch_supported(int nu, int tu) { return nu >= 1 && nu <= 4 && (tu == 16 || tu == 32); }
// The persistent launch's bounded wait on purpose: one task whose
// prerequisite segment has no task in the queue, so its counter never
// reaches the segment's block count; the wait gives up and sets *cb.err.
// ws: device workspace of kCoarseWaitTestBytes bytes.
cudaError_t launch_coarse_wait_selftest(void* ws, int* err, cudaStream_t s) {
  char* b = static_cast<char*>(ws);
  CoarseSeg segs[2] = {{0, 0, 1, -1, 0}, {0, 0, 1, 0, 0}};
  const int2 task = make_int2(1, 0);
  cudaError_t e = cudaMemcpyAsync(b, segs, sizeof(segs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + 256, &task, sizeof(task), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + 512, 0, 3 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  CoarseBatch cb{};
  cb.seg = reinterpret_cast<const CoarseSeg*>(b);
  cb.task = reinterpret_cast<const int2*>(b + 256);
  cb.ntasks = 1;
  cb.ra = nullptr;  // never reached: the only task gives up before its body
  cb.ua = nullptr;
  cb.head = reinterpret_cast<unsigned*>(b + 512);
  cb.done = cb.head + 1;
  cb.err = err;
  k_coarse_batch<3, 32><<<1, UNT, upwind_smem<float, 3, 32>(), s>>>(cb);
  return cudaGetLastError();
}
cudaError_t launch_coarse_batch(const CoarseBatch& cb, int nu, int tu, int ctas, cudaStream_t s) {
  const bool t32 = tu == 32;
  switch (nu) {
    case 1: return t32 ? launch_cb<1, 32>(cb, ctas, s) : launch_cb<1, 16>(cb, ctas, s);
    case 2: return t32 ? launch_cb<2, 32>(cb, ctas, s) : launch_cb<2, 16>(cb, ctas, s);
    case 3: return t32 ? launch_cb<3, 32>(cb, ctas, s) : launch_cb<3, 16>(cb, ctas, s);
    case 4: return t32 ? launch_cb<4, 32>(cb, ctas, s) : launch_cb<4, 16>(cb, ctas, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sum(const double* part, int n, double* out, cudaStream_t s) {
  return launch_pdl(k_sum, dim3(1), dim3(1024), 0, s, part, n, out);
}
// restriction level 0 -> 1 of r = r' + b with the norm partials
// (k_restrict4_rb); false when the level is not of k_restrict4's form or
// the partials do not fit max_parts; *nparts receives their number
bool restrict_rb_applies(int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc, int ncc, int fx, int fy,
                         int fr, int fc, int max_parts, int* nparts) {
  if (!(fx == 2 && fy == 2 && fr == 2 && fc == 2 && nx == 2 * nxc && ny == 2 * nyc && nr == 2 * nrc &&
        nc == 2 * ncc && nxc % 4 == 0 && 8 * nrc * ncc <= 65535))
    return false;
  const long parts = (long)((nxc / 4 + 31) / 32) * ((nyc + 7) / 8) * (8 * nrc * ncc);
  if (parts > max_parts) return false;
  *nparts = (int)parts;
  return true;
}
cudaError_t launch_restrict_rb(float* r, const float* b, float* coarse, const float* rcoef, const Dir<float>* dir,
                               double dxdy, double* part, int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc,
                               int ncc, cudaStream_t s) {
  const dim3 block(32, 8), grid((nxc / 4 + 31) / 32, (nyc + 7) / 8, 8 * nrc * ncc);
  return launch_pdl(k_restrict4_rb, grid, block, 0, s, r, b, coarse, rcoef, dir, dxdy, part, nx, ny, nr, nc, nxc,
                    nyc, nrc, ncc);
}
cudaError_t launch_sum2(const double* part_a, int na, double* out_a, const double* part_b, int nb, double* out_b,
                        cudaStream_t s) {
  return launch_pdl(k_sum2, dim3(1), dim3(1024), 0, s, part_a, na, out_a, part_b, nb, out_b);
}
#endif


}  // namespace btmg
