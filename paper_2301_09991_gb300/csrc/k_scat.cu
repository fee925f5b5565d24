// k_scat.cu -- the scattering smoother: a variant of the upwind correction
// sweeps (Eq. matrix_full with beta = 1, upwind filters of Sec. 2.4) in
// which the directions of a node are solved together with their in-node
// isotropic scattering sigma_s phi / (4 pi) (Sec. 2.2), the upstream
// neighbours taken from the previous iterate (node-block Jacobi).  The
// method as published keeps scattering out of the correction operators; the
// variant carries it on the levels of the coarsest angular resolution or on
// every level, where in-group scattering dominates.
//
// With a_n the plain Jacobi update of direction n and d_n = |mu|/dX +
// |nu|/dY + sigma_t its diagonal, the node's system is the identity plus a
// rank-one term and is solved exactly:
//   delta_n = a_n + c / d_n,   c = w sum_m p_m a_m,
//   w = kappa / (1 - kappa sum_m p_m / d_m),   kappa = sigma_s / (4 pi).
// w depends only on the level's directions and materials (k_scat_gain, once
// per problem).  A sweep stores J = a and the partial sums of p_n J_n over
// its chunk of directions; the isotropic field c is formed from the
// partials after the sweep (k_scat_corr) and applied on the fly where the
// next sweep reads its upstream values, and by the final pass
// (k_scat_final), which writes delta or, on the finest level, the update
// psi + delta with the scalar-flux partials of the result.
//
// Layout: one thread per node of a 32 x 8 tile, looping over the directions
// of its chunk; consecutive threads read consecutive x (coalesced), the
// upstream row is mostly read by the same block (L1).
#include <type_traits>

#include "btmg_common.cuh"

namespace btmg {
namespace {

constexpr int SX = 32, SY = 8;

__device__ __forceinline__ float srcp(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double srcp(double v) { return 1.0 / v; }

// Node of this thread, its four neighbours clamped into the domain (an
// out-of-domain neighbour points at the node itself: the adjacent interior
// node of the halo rule) and which of them left the domain.
struct NodeGeo {
  int x, y;
  bool in;
  size_t i0, ixm, ixp, iym, iyp;
  bool oxm, oxp, oym, oyp;
  __device__ NodeGeo(int nx, int ny, int tile) {
    const int tiles_x = (nx + SX - 1) / SX;
    x = (tile % tiles_x) * SX + threadIdx.x;
    y = (tile / tiles_x) * SY + threadIdx.y;
    in = x < nx && y < ny;
    const int xi = min(x, nx - 1), yi = min(y, ny - 1);
    oxm = xi == 0;
    oxp = xi == nx - 1;
    oym = yi == 0;
    oyp = yi == ny - 1;
    i0 = (size_t)yi * nx + xi;
    ixm = oxm ? i0 : i0 - 1;
    ixp = oxp ? i0 : i0 + 1;
    iym = oym ? i0 : i0 - nx;
    iyp = oyp ? i0 : i0 + nx;
  }
};

// IM: how the previous iterate is read (INIT_SAME: J + c / d of the last
// sweep; INIT_UPSAMPLE: the coarser level's delta; INIT_ZERO: 0).  Both
// neighbours in x and in y are loaded whatever the signs of mu and nu (the
// extra ones hit L1), so no load address waits for the direction table and
// the loads of several directions are in flight together.  Grid: tiles x
// direction chunks.
constexpr int kSweepBlocksPerSM = 5;
template <typename C, int IM> __device__ __forceinline__ void sweep_item(const ScatArgs<C>& a, int tile, int chunk) {
  const NodeGeo g(a.nx, a.ny, tile);
  // distinct buffers (ping-pong): restrict lets the loads of the next
  // directions move above this direction's store
  const C* __restrict__ src = a.src;
  const C* __restrict__ jin = a.jin;
  const C* __restrict__ coarse = a.coarse;
  C* __restrict__ jout = a.jout;
  const size_t npix = (size_t)a.nx * a.ny;
  const int n_begin = chunk * a.dpc, n_end = min(n_begin + a.dpc, a.nd);
  // materials and the isotropic correction of the previous sweep at the
  // node and its neighbours (scalars: the upstream pair is chosen per
  // direction by select, not by indexing)
  const C s0 = a.sig[g.i0];
  const C sxm = a.sig[g.ixm], sxq = a.sig[g.ixp], sym = a.sig[g.iym], syq = a.sig[g.iyp];
  C cxm = C(0), cxq = C(0), cym = C(0), cyq = C(0);
  if (IM == INIT_SAME && a.cin) cxm = a.cin[g.ixm], cxq = a.cin[g.ixp], cym = a.cin[g.iym], cyq = a.cin[g.iyp];
  size_t oxm = 0, oxq = 0, oym = 0, oyq = 0;  // UpSamp parents of the neighbours
  if (IM == INIT_UPSAMPLE) {
    auto parent_of = [&](size_t i) {
      const int px = (int)(i % a.nx), py = (int)(i / a.nx);
      return (size_t)(py / a.fy) * a.nxc + px / a.fx;
    };
    oxm = parent_of(g.ixm), oxq = parent_of(g.ixp), oym = parent_of(g.iym), oyq = parent_of(g.iyp);
  }
  const size_t npixc = (size_t)a.nxc * a.nyc;
  // vacuum incoming sides of this node: the upstream value is 0 there
  const bool zxm = g.oxm && a.bc.xlo == BC_VACUUM, zxp = g.oxp && a.bc.xhi == BC_VACUUM;
  const bool zym = g.oym && a.bc.ylo == BC_VACUUM, zyp = g.oyp && a.bc.yhi == BC_VACUUM;
  C acc = C(0);
#pragma unroll 4
  for (int n = n_begin; n < n_end; ++n) {
    C vxm = C(0), vxp = C(0), vym = C(0), vyp = C(0);
    if (IM == INIT_SAME) {
      const C* jn = jin + (size_t)n * npix;
      vxm = jn[g.ixm], vxp = jn[g.ixp], vym = jn[g.iym], vyp = jn[g.iyp];
    } else if (IM == INIT_UPSAMPLE) {
      const C* cn = coarse + (size_t)a.parent[n] * npixc;
      vxm = cn[oxm], vxp = cn[oxq], vym = cn[oym], vyp = cn[oyq];
    }
    const C sv = src[(size_t)n * a.src_stride + g.i0];
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    C ux = sxp ? vxm : vxp, uy = syp ? vym : vyp;
    if (IM == INIT_SAME) {
      ux += (sxp ? cxm : cxq) * srcp(dr.ax + dr.ay + (sxp ? sxm : sxq));
      uy += (syp ? cym : cyq) * srcp(dr.ax + dr.ay + (syp ? sym : syq));
    }
    if (sxp ? zxm : zxp) ux = C(0);
    if (syp ? zym : zyp) uy = C(0);
    const C J = (sv + dr.ax * ux + dr.ay * uy) * srcp(dr.ax + dr.ay + s0);
    if (g.in) jout[(size_t)n * npix + g.i0] = J;
    acc += dr.w * J;
  }
  if (g.in) a.part[(size_t)chunk * npix + g.i0] = acc;
}

template <typename C, int IM>
__global__ void __launch_bounds__(SX * SY, kSweepBlocksPerSM) k_scat_sweep(const ScatArgs<C> a) {
  sweep_item<C, IM>(a, blockIdx.x, blockIdx.y);
}

// FP32 sweeps from J + c / d (sweeps 2..nu) with four consecutive nodes per
// thread (128 x 8 node tiles): 128-bit loads of the node's row, of the rows
// above and below and of the source, the x-upstream values from the
// neighbouring lanes (warp-edge lanes load theirs), so a thread has four
// times the bytes in flight of the one-node sweep.  Needs nx % 4 == 0.
constexpr int VX = 4 * SX;
__global__ void __launch_bounds__(SX * SY, 3) k_scat_sweep_v4(const ScatArgs<float> a) {
  const int tiles_x = (a.nx + VX - 1) / VX;
  const int nx = a.nx, ny = a.ny;
  const int tx = threadIdx.x;
  int x0 = (blockIdx.x % tiles_x) * VX + 4 * tx;
  int y = (blockIdx.x / tiles_x) * SY + threadIdx.y;
  const bool in = x0 < nx && y < ny;
  x0 = min(x0, nx - 4);  // inactive lanes read in-domain values and store nothing
  y = min(y, ny - 1);
  const size_t npix = (size_t)nx * ny;
  const size_t r0 = (size_t)y * nx + x0;
  const size_t rm = y > 0 ? r0 - nx : r0, rp = y < ny - 1 ? r0 + nx : r0;
  const size_t il = x0 > 0 ? r0 - 1 : r0, ir = x0 + 4 < nx ? r0 + 4 : r0 + 3;
  const bool zl = x0 == 0 && a.bc.xlo == BC_VACUUM, zr = x0 + 4 >= nx && a.bc.xhi == BC_VACUUM;
  const bool zym = y == 0 && a.bc.ylo == BC_VACUUM, zyp = y == ny - 1 && a.bc.yhi == BC_VACUUM;
  auto ld4g = [](const float* p) { return *reinterpret_cast<const float4*>(p); };
  const float4 sg = ld4g(a.sig + r0), sgm = ld4g(a.sig + rm), sgp = ld4g(a.sig + rp);
  const float sgl = a.sig[il], sgr = a.sig[ir];
  float4 cc = make_float4(0.f, 0.f, 0.f, 0.f), ccm = cc, ccp = cc;
  float ccl = 0.f, ccr = 0.f;
  if (a.cin) cc = ld4g(a.cin + r0), ccm = ld4g(a.cin + rm), ccp = ld4g(a.cin + rp), ccl = a.cin[il], ccr = a.cin[ir];
  const float* __restrict__ src = a.src;
  const float* __restrict__ jin = a.jin;
  float* __restrict__ jout = a.jout;
  const int chunk = blockIdx.y;
  const int n_begin = chunk * a.dpc, n_end = min(n_begin + a.dpc, a.nd);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<float> dr = a.dir[n];  // uniform: one load per warp, ahead of the row loads
    const bool sxp = dr.mu > 0.f, syp = dr.nu > 0.f;
    const float* jn = jin + (size_t)n * npix;
    const float4 v = ld4g(jn + r0), vy = ld4g(jn + (syp ? rm : rp));  // own row, upstream row
    const float4 sv = ld4g(src + (size_t)n * a.src_stride + r0);
    float left = __shfl_up_sync(0xffffffffu, v.w, 1), right = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (tx == 0 || x0 == 0) left = jn[il];   // warp edge, or the node itself at the boundary
    if (tx == SX - 1 || x0 + 4 >= nx) right = jn[ir];
    const float dd = dr.ax + dr.ay;
    const float vv[4] = {v.x, v.y, v.z, v.w}, sgv[4] = {sg.x, sg.y, sg.z, sg.w}, ssv[4] = {sv.x, sv.y, sv.z, sv.w};
    const float yv[4] = {vy.x, vy.y, vy.z, vy.w};
    const float yc[4] = {syp ? ccm.x : ccp.x, syp ? ccm.y : ccp.y, syp ? ccm.z : ccp.z, syp ? ccm.w : ccp.w};
    const float ys[4] = {syp ? sgm.x : sgp.x, syp ? sgm.y : sgp.y, syp ? sgm.z : sgp.z, syp ? sgm.w : sgp.w};
    const float cv[4] = {cc.x, cc.y, cc.z, cc.w};
    const bool zy = syp ? zym : zyp;
    float J[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // x-upstream node: k - 1 (mu > 0) or k + 1, the lane neighbours at the ends
      float ux, cx, sx;
      if (sxp) {
        ux = k == 0 ? left : vv[k - 1];
        cx = k == 0 ? ccl : cv[k - 1];
        sx = k == 0 ? sgl : sgv[k - 1];
      } else {
        ux = k == 3 ? right : vv[k + 1];
        cx = k == 3 ? ccr : cv[k + 1];
        sx = k == 3 ? sgr : sgv[k + 1];
      }
      ux += cx * srcp(dd + sx);
      if (sxp ? (k == 0 && zl) : (k == 3 && zr)) ux = 0.f;
      float uy = yv[k] + yc[k] * srcp(dd + ys[k]);
      if (zy) uy = 0.f;
      J[k] = (ssv[k] + dr.ax * ux + dr.ay * uy) * srcp(dd + sgv[k]);
      acc[k] += dr.w * J[k];
    }
    if (in) *reinterpret_cast<float4*>(jout + (size_t)n * npix + r0) = make_float4(J[0], J[1], J[2], J[3]);
  }
  if (in) *reinterpret_cast<float4*>(a.part + (size_t)chunk * npix + r0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// FP32 first sweep from the UpSamp of the coarser correction with four
// consecutive nodes per thread: a node pair shares its coarse parent (the
// level coarsens by 2 in x and y), so each of the three rows takes one
// 64-bit load of the coarse plane.  Needs nx % 4 == 0 and fx = fy = 2.
__global__ void __launch_bounds__(SX * SY, 3) k_scat_sweep_v4_up(const ScatArgs<float> a) {
  const int tiles_x = (a.nx + VX - 1) / VX;
  const int nx = a.nx, ny = a.ny;
  const int tx = threadIdx.x;
  int x0 = (blockIdx.x % tiles_x) * VX + 4 * tx;
  int y = (blockIdx.x / tiles_x) * SY + threadIdx.y;
  const bool in = x0 < nx && y < ny;
  x0 = min(x0, nx - 4);
  y = min(y, ny - 1);
  const size_t npix = (size_t)nx * ny, npixc = (size_t)a.nxc * a.nyc;
  const size_t r0 = (size_t)y * nx + x0;
  const int xc = x0 / 2;  // even
  const size_t c0 = (size_t)(y / 2) * a.nxc + xc;
  const size_t cm = (size_t)((y > 0 ? y - 1 : y) / 2) * a.nxc + xc;
  const size_t cp = (size_t)((y < ny - 1 ? y + 1 : y) / 2) * a.nxc + xc;
  const size_t cl = x0 > 0 ? c0 - 1 : c0, cr = x0 + 4 < nx ? c0 + 2 : c0 + 1;
  const bool zl = x0 == 0 && a.bc.xlo == BC_VACUUM, zr = x0 + 4 >= nx && a.bc.xhi == BC_VACUUM;
  const bool zym = y == 0 && a.bc.ylo == BC_VACUUM, zyp = y == ny - 1 && a.bc.yhi == BC_VACUUM;
  const float4 sg = *reinterpret_cast<const float4*>(a.sig + r0);
  const float sgv[4] = {sg.x, sg.y, sg.z, sg.w};
  const float* __restrict__ src = a.src;
  const float* __restrict__ coarse = a.coarse;
  float* __restrict__ jout = a.jout;
  const int chunk = blockIdx.y;
  const int n_begin = chunk * a.dpc, n_end = min(n_begin + a.dpc, a.nd);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
  for (int n = n_begin; n < n_end; ++n) {
    const float* cn = coarse + (size_t)a.parent[n] * npixc;
    const float2 v = *reinterpret_cast<const float2*>(cn + c0);
    const float2 vm = *reinterpret_cast<const float2*>(cn + cm);
    const float2 vp = *reinterpret_cast<const float2*>(cn + cp);
    const float4 sv = *reinterpret_cast<const float4*>(src + (size_t)n * a.src_stride + r0);
    float left = __shfl_up_sync(0xffffffffu, v.y, 1), right = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (tx == 0 || x0 == 0) left = cn[cl];  // warp edge, or the node itself at the boundary
    if (tx == SX - 1 || x0 + 4 >= nx) right = cn[cr];
    const Dir<float> dr = a.dir[n];
    const bool sxp = dr.mu > 0.f, syp = dr.nu > 0.f;
    const float dd = dr.ax + dr.ay;
    const float vv[4] = {v.x, v.x, v.y, v.y}, ssv[4] = {sv.x, sv.y, sv.z, sv.w};
    const float2 yr = syp ? vm : vp;
    const float yv[4] = {yr.x, yr.x, yr.y, yr.y};
    const bool zy = syp ? zym : zyp;
    float J[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float ux = sxp ? (k == 0 ? left : vv[k - 1]) : (k == 3 ? right : vv[k + 1]);
      if (sxp ? (k == 0 && zl) : (k == 3 && zr)) ux = 0.f;
      const float uy = zy ? 0.f : yv[k];
      J[k] = (ssv[k] + dr.ax * ux + dr.ay * uy) * srcp(dd + sgv[k]);
      acc[k] += dr.w * J[k];
    }
    if (in) *reinterpret_cast<float4*>(jout + (size_t)n * npix + r0) = make_float4(J[0], J[1], J[2], J[3]);
  }
  if (in) *reinterpret_cast<float4*>(a.part + (size_t)chunk * npix + r0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

template <typename C>
__global__ void k_scat_corr(const C* __restrict__ part, int nchunk, const C* __restrict__ w, int npix,
                            C* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  C s = C(0);
  for (int k = 0; k < nchunk; ++k) s += part[(size_t)k * npix + i];
  c[i] = w[i] * s;
}

template <typename T, typename C, bool UPDATE> __global__ void __launch_bounds__(SX * SY) k_scat_final(const ScatFinal<T, C> f) {
  const NodeGeo g(f.nx, f.ny, blockIdx.x);
  if (!g.in) return;
  const size_t npix = (size_t)f.nx * f.ny;
  const int chunk = blockIdx.y;
  const int n_begin = chunk * f.dpc, n_end = min(n_begin + f.dpc, f.nd);
  const C c0 = f.c[g.i0], s0 = f.sig[g.i0];
  C acc = C(0);
#pragma unroll 4
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<C> dr = f.dir[n];
    const size_t gi = (size_t)n * npix + g.i0;
    const C d = f.j[gi] + c0 * srcp(dr.ax + dr.ay + s0);
    if (UPDATE) {
      const C pn = (C)Conv<T>::ld(f.psi_in + gi) + d;
      Conv<T>::st(f.psi_out + gi, pn);
      acc += dr.w * stored<T, C>(pn);
    } else {
      f.delta_out[gi] = d;
    }
  }
  if (UPDATE) f.phi_part[(size_t)chunk * npix + g.i0] = acc;
}

// FP32 final pass with four consecutive nodes per thread (128-bit loads and
// stores of J and psi).  Needs nx % 4 == 0.
template <bool UPDATE> __global__ void __launch_bounds__(SX * SY) k_scat_final_v4(const ScatFinal<float, float> f) {
  const int tiles_x = (f.nx + VX - 1) / VX;
  const int x0 = (blockIdx.x % tiles_x) * VX + 4 * threadIdx.x;
  const int y = (blockIdx.x / tiles_x) * SY + threadIdx.y;
  if (x0 >= f.nx || y >= f.ny) return;
  const size_t npix = (size_t)f.nx * f.ny, r0 = (size_t)y * f.nx + x0;
  const int chunk = blockIdx.y;
  const int n_begin = chunk * f.dpc, n_end = min(n_begin + f.dpc, f.nd);
  const float4 c4 = *reinterpret_cast<const float4*>(f.c + r0);
  const float4 s4 = *reinterpret_cast<const float4*>(f.sig + r0);
  const float cv[4] = {c4.x, c4.y, c4.z, c4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<float> dr = f.dir[n];
    const size_t gi = (size_t)n * npix + r0;
    const float4 j4 = *reinterpret_cast<const float4*>(f.j + gi);
    const float jv[4] = {j4.x, j4.y, j4.z, j4.w};
    float d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = jv[k] + cv[k] * srcp(dr.ax + dr.ay + sv[k]);
    if (UPDATE) {
      const float4 p4 = *reinterpret_cast<const float4*>(f.psi_in + gi);
      const float pn[4] = {p4.x + d[0], p4.y + d[1], p4.z + d[2], p4.w + d[3]};
      *reinterpret_cast<float4*>(f.psi_out + gi) = make_float4(pn[0], pn[1], pn[2], pn[3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += dr.w * pn[k];
    } else {
      *reinterpret_cast<float4*>(f.delta_out + gi) = make_float4(d[0], d[1], d[2], d[3]);
    }
  }
  if (UPDATE)
    *reinterpret_cast<float4*>(f.phi_part + (size_t)chunk * npix + r0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

template <typename C>
__global__ void k_scat_gain(const C* __restrict__ sig, const C* __restrict__ crat, const Dir<C>* __restrict__ dir,
                            int nd, int npix, C* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const double st = (double)sig[i];
  double S = 0.0;
  for (int n = 0; n < nd; ++n) S += (double)dir[n].w / ((double)dir[n].ax + (double)dir[n].ay + st);
  const double kappa = (double)crat[i] * st / (4.0 * 3.14159265358979323846);
  w[i] = (C)(kappa / (1.0 - kappa * S));
}

// Division by a run-time divisor d in [1, 2^16) of a numerator x in
// [0, 2^16) as one multiply-high: with m = ceil(2^32 / d) the error
// x (m - 2^32/d) / 2^32 < 2^-16 <= 1/d never carries past the next integer,
// so the quotient is exact.
struct FDiv {
  uint32_t m;
  int d;
  __device__ __forceinline__ explicit FDiv(int dd) : m(dd > 1 ? 0xFFFFFFFFu / (uint32_t)dd + 1u : 0u), d(dd) {}
  __device__ __forceinline__ int div(int x) const { return d == 1 ? x : (int)__umulhi((uint32_t)x, m); }
};

// The small coarsest levels in one CTA (as separate kernels they are
// launch-bound): the restrictions down these levels (the restriction of
// Sec. 2.5 as k_restrict computes it), then for each level from the
// coarsest up nu sweeps and the final pass with block barriers between the
// phases; the sweep iterates, the isotropic field and the coarser level's
// correction live in shared memory.  SCAT = false: the published upwind
// Jacobi (delta = J of the last sweep); SCAT = true: the scattering
// smoother, its scalar flux summed over all directions at once.
template <typename C, int TMAX, bool SCAT> __global__ void __launch_bounds__(1024) k_tail(const ScatTail<C> t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();
  pdl_launch();
  C* Ja = reinterpret_cast<C*>(smem_raw);
  C* Jb = Ja + TMAX;
  C* Dc = Jb + TMAX;  // the coarser level's delta, then this level's
  C* cf = Dc + TMAX;  // isotropic correction c of the last sweep, [ny][nx]
  for (int li = 0; li + 1 < t.count; ++li) {
    const ScatTailLevel<C> F = t.lev[li], Q = t.lev[li + 1];
    const int total = Q.nd * Q.ny * Q.nx;
    const FDiv dnx(Q.nx), dny(Q.ny), dnrc(Q.nr * Q.nc), dnc(Q.nc);
#pragma unroll 4
    for (int id = threadIdx.x; id < total; id += blockDim.x) {
      const int idy = dnx.div(id), N = dny.div(idy);
      const int X = id - idy * Q.nx, Y = idy - N * Q.ny;
      const int f = dnrc.div(N), Jn = N - f * Q.nr * Q.nc, J = dnc.div(Jn), I = Jn - J * Q.nc;
      C acc = C(0);
      for (int aa = 0; aa < F.fr; ++aa) {
        const int j = J * F.fr + aa;
        if (j >= F.nr) continue;
        for (int bb = 0; bb < F.fc; ++bb) {
          const int i = I * F.fc + bb;
          if (i >= F.nc) continue;
          const int n = f * F.nr * F.nc + j * F.nc + i;
          const C w = F.rcoef[n];
          for (int yy = 0; yy < F.fy; ++yy) {
            const int y = Y * F.fy + yy;
            if (y >= F.ny) continue;
            for (int xx = 0; xx < F.fx; ++xx) {
              const int x = X * F.fx + xx;
              if (x >= F.nx) continue;
              acc += w * F.s[(n * F.ny + y) * F.nx + x];
            }
          }
        }
      }
      Q.s[id] = acc;
    }
    __syncthreads();
  }
  for (int li = t.count - 1; li >= 0; --li) {
    const ScatTailLevel<C> L = t.lev[li];
    const C* __restrict__ ls = L.s;
    const C* __restrict__ lsig = L.sig;
    const int npix = L.nx * L.ny, n_all = npix * L.nd;
    const bool has_coarse = li + 1 < t.count;
    const int nxc = has_coarse ? t.lev[li + 1].nx : 1, npixc = has_coarse ? nxc * t.lev[li + 1].ny : 1;
    const FDiv dpix(npix), dx(L.nx), dfy(L.fy), dfx(L.fx);
    C* Jprev = nullptr;
    C* Jcur = Ja;
    for (int k = 1; k <= t.nu; ++k) {
#pragma unroll 4
      for (int idx = threadIdx.x; idx < n_all; idx += blockDim.x) {
        const int dn = dpix.div(idx), i = idx - dn * npix;
        const int y = dx.div(i), x = i - y * L.nx;
        const Dir<C> dr = L.dir[dn];
        const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
        int xu = sxp ? x - 1 : x + 1, yu = syp ? y - 1 : y + 1;
        const bool outx = xu < 0 || xu >= L.nx, outy = yu < 0 || yu >= L.ny;
        const bool zx = outx && (sxp ? t.bc.xlo : t.bc.xhi) == BC_VACUUM;
        const bool zy = outy && (syp ? t.bc.ylo : t.bc.yhi) == BC_VACUUM;
        if (outx) xu = x;  // reflective: the adjacent interior node
        if (outy) yu = y;
        const int ix = y * L.nx + xu, iy = yu * L.nx + x;
        C ux = C(0), uy = C(0);
        if (k > 1) {
          if (!zx) ux = Jprev[dn * npix + ix];
          if (!zy) uy = Jprev[dn * npix + iy];
          if (SCAT) {
            if (!zx) ux += cf[ix] * srcp(dr.ax + dr.ay + L.sig[ix]);
            if (!zy) uy += cf[iy] * srcp(dr.ax + dr.ay + L.sig[iy]);
          }
        } else if (has_coarse) {
          const C* cn = Dc + L.parent[dn] * npixc;
          if (!zx) ux = cn[dfy.div(y) * nxc + dfx.div(xu)];
          if (!zy) uy = cn[dfy.div(yu) * nxc + dfx.div(x)];
        }
        Jcur[idx] = (ls[idx] + dr.ax * ux + dr.ay * uy) * srcp(dr.ax + dr.ay + lsig[i]);
      }
      __syncthreads();
      if (SCAT) {
        for (int i = threadIdx.x; i < npix; i += blockDim.x) {
          C sum = C(0);
          for (int dn = 0; dn < L.nd; ++dn) sum += L.dir[dn].w * Jcur[dn * npix + i];
          cf[i] = L.w[i] * sum;
        }
        __syncthreads();
      }
      Jprev = Jcur;
      Jcur = Jcur == Ja ? Jb : Ja;
    }
#pragma unroll 4
    for (int idx = threadIdx.x; idx < n_all; idx += blockDim.x) {
      C d = Jprev[idx];
      if (SCAT) {
        const int dn = dpix.div(idx), i = idx - dn * npix;
        const Dir<C> dr = L.dir[dn];
        d += cf[i] * srcp(dr.ax + dr.ay + L.sig[i]);
      }
      if (li == 0)
        t.out[idx] = d;
      else
        Dc[idx] = d;
    }
    __syncthreads();
  }
}

// 16-byte aligned (or absent) buffer: the four-node kernels use 128-bit accesses
bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

dim3 node_grid(int nx, int ny, int nchunk) {
  return dim3(((nx + SX - 1) / SX) * ((ny + SY - 1) / SY), nchunk);
}

}  // namespace

template <typename C> cudaError_t launch_scat_sweep(const ScatArgs<C>& a, int nchunk, cudaStream_t s) {
  const dim3 grid = node_grid(a.nx, a.ny, nchunk), block(SX, SY);
  if constexpr (sizeof(C) == 4) {
    if (a.init_mode == INIT_SAME && scat_vec(a.nx, 4) && al16(a.src) && al16(a.jin) && al16(a.jout) &&
        al16(a.cin) && al16(a.part) && al16(a.sig)) {
      const dim3 g4(((a.nx + VX - 1) / VX) * ((a.ny + SY - 1) / SY), nchunk);
      k_scat_sweep_v4<<<g4, block, 0, s>>>(a);
      return cudaGetLastError();
    }
    if (a.init_mode == INIT_UPSAMPLE && scat_vec(a.nx, 4) && a.fx == 2 && a.fy == 2 && al16(a.src) &&
        al16(a.jout) && al16(a.part) && al16(a.sig) && ((uintptr_t)a.coarse & 7u) == 0) {
      const dim3 g4(((a.nx + VX - 1) / VX) * ((a.ny + SY - 1) / SY), nchunk);
      k_scat_sweep_v4_up<<<g4, block, 0, s>>>(a);
      return cudaGetLastError();
    }
  }
  if (a.init_mode == INIT_SAME)
    k_scat_sweep<C, INIT_SAME><<<grid, block, 0, s>>>(a);
  else if (a.init_mode == INIT_UPSAMPLE)
    k_scat_sweep<C, INIT_UPSAMPLE><<<grid, block, 0, s>>>(a);
  else
    k_scat_sweep<C, INIT_ZERO><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename C>
cudaError_t launch_scat_corr(const C* part, int nchunk, const C* w, int npix, C* c, cudaStream_t s) {
  k_scat_corr<C><<<(npix + 255) / 256, 256, 0, s>>>(part, nchunk, w, npix, c);
  return cudaGetLastError();
}

template <typename T, typename C> cudaError_t launch_scat_final(const ScatFinal<T, C>& f, int nchunk, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value && std::is_same<C, float>::value) {
    if (scat_vec(f.nx, 4) && al16(f.j) && al16(f.c) && al16(f.sig) && al16(f.psi_in) && al16(f.psi_out) &&
        al16(f.delta_out) && al16(f.phi_part)) {
      const dim3 g4(((f.nx + VX - 1) / VX) * ((f.ny + SY - 1) / SY), nchunk);
      if (f.psi_out)
        k_scat_final_v4<true><<<g4, dim3(SX, SY), 0, s>>>(f);
      else
        k_scat_final_v4<false><<<g4, dim3(SX, SY), 0, s>>>(f);
      return cudaGetLastError();
    }
  }
  if (f.psi_out)
    k_scat_final<T, C, true><<<node_grid(f.nx, f.ny, nchunk), dim3(SX, SY), 0, s>>>(f);
  else
    k_scat_final<T, C, false><<<node_grid(f.nx, f.ny, nchunk), dim3(SX, SY), 0, s>>>(f);
  return cudaGetLastError();
}

template <typename C>
cudaError_t launch_scat_gain(const C* sig, const C* crat, const Dir<C>* dir, int nd, int npix, C* w, cudaStream_t s) {
  k_scat_gain<C><<<(npix + 255) / 256, 256, 0, s>>>(sig, crat, dir, nd, npix, w);
  return cudaGetLastError();
}

template <typename C, bool SCAT> cudaError_t launch_tail_mode(const ScatTail<C>& t, cudaStream_t s) {
  constexpr int TMAX = scat_tail_max<C>();
  constexpr size_t smem = (3 * (size_t)TMAX + TMAX / 8) * sizeof(C);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tail<C, TMAX, SCAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return launch_pdl(k_tail<C, TMAX, SCAT>, dim3(1), dim3(1024), smem, s, t);
}
template <typename C> cudaError_t launch_scat_tail(const ScatTail<C>& t, cudaStream_t s) {
  return t.scat ? launch_tail_mode<C, true>(t, s) : launch_tail_mode<C, false>(t, s);
}

// node-tile chunking shared by the sweep launches and the workspace sizing
bool scat_vec(int nx, int csize) { return csize == 4 && nx % 4 == 0; }

int scat_chunks(int nx, int ny, int nd, int csize) {
  const int tw = scat_vec(nx, csize) ? VX : SX;  // node tile width of the sweeps from J
  const int tiles = ((nx + tw - 1) / tw) * ((ny + SY - 1) / SY);
  const int want = (2432 + tiles - 1) / tiles;  // about 16 blocks per SM over the launch
  int c = want < 1 ? 1 : (want > 64 ? 64 : want);
  if (c > nd) c = nd;
  const int dpc = (nd + c - 1) / c;
  return (nd + dpc - 1) / dpc;
}

#define INST_SC(C)                                                                                       \
  template cudaError_t launch_scat_sweep<C>(const ScatArgs<C>&, int, cudaStream_t);                      \
  template cudaError_t launch_scat_corr<C>(const C*, int, const C*, int, C*, cudaStream_t);              \
  template cudaError_t launch_scat_gain<C>(const C*, const C*, const Dir<C>*, int, int, C*, cudaStream_t); \
  template cudaError_t launch_scat_tail<C>(const ScatTail<C>&, cudaStream_t);
INST_SC(double)
INST_SC(float)
template cudaError_t launch_scat_final<double, double>(const ScatFinal<double, double>&, int, cudaStream_t);
template cudaError_t launch_scat_final<float, float>(const ScatFinal<float, float>&, int, cudaStream_t);
template cudaError_t launch_scat_final<__nv_bfloat16, float>(const ScatFinal<__nv_bfloat16, float>&, int,
                                                              cudaStream_t);
template cudaError_t launch_scat_final<__half, float>(const ScatFinal<__half, float>&, int, cudaStream_t);

}  // namespace btmg
