// k_upres.cu -- fine-level residual and Jacobi sweep of the upwind scheme
// (pg = 0: the upwind filters of Sec. 2.4 on the finest level, Eq. matrix_full
// with beta = 1), as a streaming kernel.
//
//   r   = b + extra - (mu u_x / dx + nu u_y / dy + sigma_t psi)
//   u_x = psi(x) - psi(x - 1) for mu > 0, psi(x + 1) - psi(x) for mu < 0
//   (u_y likewise), the out-of-domain neighbour following the halo rule of
//   Sec. 2.3 (the upstream side is always incoming: 0 on a vacuum side, the
//   boundary node itself on a reflective side);
//   RESID:  r out, sum_n p_n r (rho partials), sum p dx dy r^2 (FP64);
//   JACOBI: psi_out = psi + r / (beta (|mu|/dx + |nu|/dy + sigma_t)) and the
//   scalar-flux partials of psi_out.
//
// The stencil reaches one node upstream.  One CTA owns a 128 x 8 tile and a
// chunk of directions (the partial sums per chunk as in k_pg), a warp one
// 128-node row segment (whole 512-byte FP32 rows per access) and a thread 4
// consecutive nodes, whose sigma_t and b stay in registers across the
// directions.  Two variants:
//   k_upres_tma (the one that runs when psi's rows are 16-byte multiples):
//     per direction a 144 x 10 box around the tile arrives in shared memory
//     by one TMA copy, KS directions ahead (mbarrier pipeline, bounded
//     waits); the upstream row and the tile-edge columns are read from the
//     box, the neighbour columns inside the segment by lane shuffles;
//   k_upres (any layout): the same work with plain loads, the next
//     direction's values fetched into registers while the current one is
//     computed.
// Neither needs barriers inside a direction: the kernel streams psi in and
// r (or psi) out.
#include <cstring>
#include <type_traits>

#include "btmg_common.cuh"
#include "tma.cuh"

namespace btmg {
namespace {

// CTA tile: 128 x 8 nodes, one warp per 128-node row segment (whole 512-byte
// rows of FP32 per warp access), a thread owns 4 consecutive nodes
constexpr int RTX = 128, RTY = 8, RNT = 256;

// 4 consecutive elements (vector access when VEC: 16-byte rows of float,
// 8-byte rows of BF16/FP16, two 16-byte halves of double).
template <typename T, typename C, bool VEC> struct Quad {
  __device__ __forceinline__ static void ld(const T* p, int nv, C v[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = k < nv ? (C)Conv<T>::ld(p + k) : C(0);
  }
  __device__ __forceinline__ static void st(T* p, int nv, const C v[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < nv) Conv<T>::st(p + k, v[k]);
  }
};
template <> struct Quad<float, float, true> {
  __device__ __forceinline__ static void ld(const float* p, int nv, float v[4]) {
    if (nv == 4) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
    } else {
      Quad<float, float, false>::ld(p, nv, v);
    }
  }
  __device__ __forceinline__ static void st(float* p, int nv, const float v[4]) {
    if (nv == 4)
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
      Quad<float, float, false>::st(p, nv, v);
  }
};
template <> struct Quad<double, double, true> {
  __device__ __forceinline__ static void ld(const double* p, int nv, double v[4]) {
    if (nv == 4) {
      const double2 a = __ldg(reinterpret_cast<const double2*>(p));
      const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
      v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    } else {
      Quad<double, double, false>::ld(p, nv, v);
    }
  }
  __device__ __forceinline__ static void st(double* p, int nv, const double v[4]) {
    if (nv == 4) {
      reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
      reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    } else {
      Quad<double, double, false>::st(p, nv, v);
    }
  }
};
template <typename H> struct Quad16 {  // BF16 / FP16 storage, FP32 compute
  __device__ __forceinline__ static void ld(const H* p, int nv, float v[4]) {
    if (nv == 4) {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      const H* h = reinterpret_cast<const H*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = Conv<H>::ld(h + k);
    } else {
      Quad<H, float, false>::ld(p, nv, v);
    }
  }
  __device__ __forceinline__ static void st(H* p, int nv, const float v[4]) {
    if (nv == 4) {
      uint2 u;
      H* h = reinterpret_cast<H*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) Conv<H>::st(h + k, v[k]);
      *reinterpret_cast<uint2*>(p) = u;
    } else {
      Quad<H, float, false>::st(p, nv, v);
    }
  }
};
template <> struct Quad<__nv_bfloat16, float, true> : Quad16<__nv_bfloat16> {};
template <> struct Quad<__half, float, true> : Quad16<__half> {};

template <typename T, typename C, int MODE, bool VEC>
__global__ void __launch_bounds__(RNT, 4) k_upres(const PgArgs<T, C> a) {
  __shared__ double red[RNT / 32];
  pdl_wait();
  pdl_launch();
  const int tid = threadIdx.x;
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int tiles_sx = (a.nx + RTX - 1) / RTX;
  const int x0 = (tile % tiles_sx) * RTX, y0 = (tile / tiles_sx) * RTY;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;
  const int q = tid & 31;  // a warp holds one 128-node row segment, lane q its quad q
  const int gy = y0 + (tid >> 5), gx = x0 + 4 * q;
  const int nv = gy < ny ? max(0, min(4, nx - gx)) : 0;  // valid nodes of this quad
  const size_t gi = (size_t)(gy < ny ? gy : 0) * nx + (gx < nx ? gx : 0);

  C sig[4], bb[4], acc[4];
  Quad<C, C, VEC>::ld(a.sigt + gi, nv, sig);
  Quad<C, C, VEC>::ld(a.b + gi, nv, bb);
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = C(0);
  double nrm = 0.0;

  const int n_begin = chunk * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);
  // this quad's values, the upstream row's and the upstream edge value for
  // direction n (loaded one direction ahead)
  C pc[4], pu[4], pe;
  auto fetch = [&](int n, C (&c)[4], C (&u)[4], C& e) {
    const Dir<C> dr = a.dir[n];
    const T* pn = a.psi + (size_t)n * npix;
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    Quad<T, C, VEC>::ld(pn + gi, nv, c);
    const int uy = syp ? gy - 1 : gy + 1;
    if (nv > 0 && uy >= 0 && uy < ny) {
      Quad<T, C, VEC>::ld(pn + (size_t)uy * nx + gx, nv, u);
    } else {
      const bool refl = syp ? a.bc.ylo == BC_REFLECTIVE : a.bc.yhi == BC_REFLECTIVE;
#pragma unroll
      for (int k = 0; k < 4; ++k) u[k] = refl ? c[k] : C(0);
    }
    // upstream column outside this quad: x0 - 1 for q = 0 (mu > 0), x0 + 128
    // for q = 31 (mu < 0); the other lanes take it from their neighbour
    e = C(0);
    if (nv > 0) {
      const int ex = sxp ? gx - 1 : gx + 4;
      if ((sxp ? q == 0 : q == 31) && ex >= 0 && ex < nx) e = (C)Conv<T>::ld(pn + (size_t)gy * nx + ex);
    }
  };
  if (n_begin < n_end) fetch(n_begin, pc, pu, pe);
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    C c[4], u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = pc[k], u[k] = pu[k];
    const C edge = pe;
    if (n + 1 < n_end) fetch(n + 1, pc, pu, pe);
    // neighbour lanes' end values (every lane takes part in the shuffles)
    const C from_left = __shfl_up_sync(0xffffffffu, c[3], 1);
    const C from_right = __shfl_down_sync(0xffffffffu, c[0], 1);
    const bool xrefl = sxp ? a.bc.xlo == BC_REFLECTIVE : a.bc.xhi == BC_REFLECTIVE;
    C out[4];
    C nrm_dir = C(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      out[k] = C(0);
      if (k >= nv) continue;
      const int xu = sxp ? gx + k - 1 : gx + k + 1;  // upstream column
      C vu;
      if (xu < 0 || xu >= nx)
        vu = xrefl ? c[k] : C(0);
      else if (sxp)
        vu = k > 0 ? c[k - 1] : (q > 0 ? from_left : edge);
      else
        vu = k < 3 ? c[k + 1] : (q < 31 ? from_right : edge);
      const C ux = sxp ? c[k] - vu : vu - c[k];
      const C uy = syp ? c[k] - u[k] : u[k] - c[k];
      const C Apsi = dr.mu * ux * a.inv_dx + dr.nu * uy * a.inv_dy + sig[k] * c[k];
      const C r = bb[k] + (a.extra ? a.extra[(size_t)n * npix + gi + k] : C(0)) - Apsi;
      if (MODE == PG_RESID) {
        out[k] = r;
        nrm_dir += r * r;
        acc[k] += dr.w * r;
      } else {
        const C d = a.beta * (dr.ax + dr.ay + sig[k]);
        out[k] = c[k] + r / d;
        acc[k] += dr.w * stored<T, C>(out[k]);
      }
    }
    if (MODE == PG_RESID) {
      Quad<C, C, VEC>::st(a.r_out + (size_t)n * npix + gi, nv, out);
      nrm += (double)dr.w * (double)nrm_dir;
    } else {
      Quad<T, C, VEC>::st(a.psi_out + (size_t)n * npix + gi, nv, out);
    }
  }
  C* part = MODE == PG_JACOBI ? a.phi_part : a.rho_part;
  if (part) Quad<C, C, VEC>::st(part + (size_t)chunk * npix + gi, nv, acc);
  if (MODE == PG_RESID) {
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) red[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < RNT / 32; ++w) s += red[w];
      a.norm_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s * (double)a.dxdy;
    }
  }
}

// TMA-staged variant.  Per direction the CTA's 128 x 8 tile plus one row
// above and below and 8 columns on each side (a 144 x 10 box starting at
// (x0 - 8, y0 - 1): the x coordinate stays a multiple of 16 bytes) arrives in
// shared memory by one cp.async.bulk.tensor copy; KS stages are in flight, so
// the loads sit in shared memory, not in registers.  Out-of-domain cells of
// the box arrive as 0 (the vacuum halo); reflective sides are resolved at
// use.  Waits on the stage barriers are bounded: on a timeout the CTA sets
// the error flag, waits (bounded) for its copies in flight and returns.
constexpr int BXS = RTX + 16, BYS = RTY + 2, KS = 4;
template <typename T> __host__ __device__ constexpr int stage_bytes() {
  return (int)(((size_t)BXS * BYS * sizeof(T) + 127) / 128 * 128);
}

template <typename T, typename C, int MODE>
__global__ void __launch_bounds__(RNT, 4) k_upres_tma(const PgArgs<T, C> a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[KS];
  __shared__ double red[RNT / 32];
  pdl_wait();
  pdl_launch();
  const int tid = threadIdx.x;
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int tiles_sx = (a.nx + RTX - 1) / RTX;
  const int x0 = (tile % tiles_sx) * RTX, y0 = (tile / tiles_sx) * RTY;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;
  const int q = tid & 31, row = tid >> 5;
  const int gy = y0 + row, gx = x0 + 4 * q;
  const int nv = gy < ny ? max(0, min(4, nx - gx)) : 0;
  const size_t gi = (size_t)(gy < ny ? gy : 0) * nx + (gx < nx ? gx : 0);
  constexpr uint32_t SB = (uint32_t)stage_bytes<T>();
  constexpr uint32_t BOX_BYTES = (uint32_t)(BXS * BYS * sizeof(T));

  C sig[4], bb[4], acc[4];
  Quad<C, C, true>::ld(a.sigt + gi, nv, sig);
  Quad<C, C, true>::ld(a.b + gi, nv, bb);
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = C(0);
  double nrm = 0.0;

  const int n_begin = chunk * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);
  const int count = max(0, n_end - n_begin);
  if (tid == 0) {
    for (int s = 0; s < KS; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < KS && s < count; ++s) {
      mbar_expect_tx(&bars[s], BOX_BYTES);
      tma_load_3d(smem_raw + s * SB, &tmap, &bars[s], x0 - 8, y0 - 1, n_begin + s);
    }
  }
  for (int it = 0; it < count; ++it) {
    const int n = n_begin + it, s = it % KS;
    const bool got = mbar_wait_bounded(&bars[s], (uint32_t)(it / KS) & 1u);
    if (!__syncthreads_and(got)) {  // the copy engine stalled: flag it, drain, leave together
      if (tid == 0) {
        atomicExch(a.err, 1);
        for (int j = it + 1; j < count && j < it + KS; ++j) mbar_wait_bounded(&bars[j % KS], (uint32_t)(j / KS) & 1u);
      }
      return;
    }
    const T* st = reinterpret_cast<const T*>(smem_raw + s * SB);
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    const T* rc = st + (row + 1) * BXS + 8 + 4 * q;  // this quad
    const T* ru = rc + (syp ? -BXS : BXS);            // the upstream row
    C c[4], vy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c[k] = (C)Conv<T>::ld(rc + k);
      vy[k] = (C)Conv<T>::ld(ru + k);
    }
    const C from_left = __shfl_up_sync(0xffffffffu, c[3], 1);
    const C from_right = __shfl_down_sync(0xffffffffu, c[0], 1);
    if (nv > 0) {  // with the vector layout a quad is full or empty
      // upstream values in x: the neighbour lane's end value, the box's
      // x0 - 1 / x0 + 128 column at the segment ends, the halo rule at the
      // domain boundary
      C vx[4];
      if (sxp) {
        vx[0] = q > 0 ? from_left : (C)Conv<T>::ld(rc - 1);
        vx[1] = c[0], vx[2] = c[1], vx[3] = c[2];
        if (gx == 0 && a.bc.xlo == BC_REFLECTIVE) vx[0] = c[0];
      } else {
        vx[0] = c[1], vx[1] = c[2], vx[2] = c[3];
        vx[3] = q < 31 ? from_right : (C)Conv<T>::ld(rc + 4);
        if (gx + 4 == nx && a.bc.xhi == BC_REFLECTIVE) vx[3] = c[3];
      }
      // the box reads 0 outside the domain (vacuum); a reflective side takes
      // the boundary node itself
      if ((syp ? gy == 0 && a.bc.ylo == BC_REFLECTIVE : gy == ny - 1 && a.bc.yhi == BC_REFLECTIVE)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) vy[k] = c[k];
      }
      // mu u_x = |mu| (psi - psi_upstream) for either sign of mu, likewise in
      // y: r = b + extra - (|mu|/dx + |nu|/dy + sigma_t) psi + |mu|/dx psi_x,up
      // + |nu|/dy psi_y,up
      C ex[4] = {C(0), C(0), C(0), C(0)};
      if (a.extra) Quad<C, C, true>::ld(a.extra + (size_t)n * npix + gi, 4, ex);
      C out[4];
      C nrm_dir = C(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const C dk = dr.ax + dr.ay + sig[k];
        const C r = bb[k] + ex[k] + dr.ax * vx[k] + dr.ay * vy[k] - dk * c[k];
        if (MODE == PG_RESID) {
          out[k] = r;
          nrm_dir += r * r;
          acc[k] += dr.w * r;
        } else {
          out[k] = c[k] + r / (a.beta * dk);
          acc[k] += dr.w * stored<T, C>(out[k]);
        }
      }
      if (MODE == PG_RESID) {
        Quad<C, C, true>::st(a.r_out + (size_t)n * npix + gi, 4, out);
        nrm += (double)dr.w * (double)nrm_dir;
      } else {
        Quad<T, C, true>::st(a.psi_out + (size_t)n * npix + gi, 4, out);
      }
    }
    __syncthreads();  // every thread is done with stage s
    if (tid == 0 && it + KS < count) {
      fence_proxy_async();
      mbar_expect_tx(&bars[s], BOX_BYTES);
      tma_load_3d(smem_raw + s * SB, &tmap, &bars[s], x0 - 8, y0 - 1, n + KS);
    }
  }
  C* part = MODE == PG_JACOBI ? a.phi_part : a.rho_part;
  if (part) Quad<C, C, true>::st(part + (size_t)chunk * npix + gi, nv, acc);
  if (MODE == PG_RESID) {
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) red[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < RNT / 32; ++w) sum += red[w];
      a.norm_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = sum * (double)a.dxdy;
    }
  }
}

template <typename T> CUtensorMapDataType tmap_type() {
  if (sizeof(T) == 8) return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  if (sizeof(T) == 4) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

template <typename T, typename C, int MODE>
cudaError_t launch_tma(const PgArgs<T, C>& a, const CUtensorMap& tm, int nchunk, cudaStream_t s) {
  constexpr int smem = KS * stage_bytes<T>();
  static bool attr_set = false;  // per instantiation, once per process
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(k_upres_tma<T, C, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid(((a.nx + RTX - 1) / RTX) * ((a.ny + RTY - 1) / RTY), nchunk);
  return launch_pdl(k_upres_tma<T, C, MODE>, grid, dim3(RNT), smem, s, a, tm);
}

bool aligned(const void* p, size_t b) { return ((uintptr_t)p % b) == 0; }

template <typename T, typename C, int MODE, bool VEC>
cudaError_t launch_v(const PgArgs<T, C>& a, int nchunk, cudaStream_t s) {
  dim3 grid(((a.nx + RTX - 1) / RTX) * ((a.ny + RTY - 1) / RTY), nchunk);
  return launch_pdl(k_upres<T, C, MODE, VEC>, grid, dim3(RNT), 0, s, a);
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_upres(const PgArgs<T, C>& a, int mode, int nchunk, cudaStream_t s) {
  // vector access needs every row to start on a 4-element boundary and the
  // buffers to be aligned to 4 elements
  const bool vec = a.nx % 4 == 0 && aligned(a.psi, 4 * sizeof(T)) && aligned(a.b, 4 * sizeof(C)) &&
                   aligned(a.sigt, 4 * sizeof(C)) && (!a.extra || aligned(a.extra, 4 * sizeof(C))) &&
                   (!a.r_out || aligned(a.r_out, 4 * sizeof(C))) &&
                   (!a.psi_out || aligned(a.psi_out, 4 * sizeof(T))) &&
                   (!a.phi_part || aligned(a.phi_part, 4 * sizeof(C))) &&
                   (!a.rho_part || aligned(a.rho_part, 4 * sizeof(C)));
  // TMA staging needs the vector layout and a tensor map over psi (16-byte
  // base and row stride); otherwise the register-pipelined kernel runs
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  if (vec && encode_tmap_3d(&tm, a.psi, tmap_type<T>(), sizeof(T), a.nx, a.ny, a.nd, BXS, BYS))
    return mode == PG_RESID ? launch_tma<T, C, PG_RESID>(a, tm, nchunk, s) : launch_tma<T, C, PG_JACOBI>(a, tm, nchunk, s);
  if (mode == PG_RESID)
    return vec ? launch_v<T, C, PG_RESID, true>(a, nchunk, s) : launch_v<T, C, PG_RESID, false>(a, nchunk, s);
  return vec ? launch_v<T, C, PG_JACOBI, true>(a, nchunk, s) : launch_v<T, C, PG_JACOBI, false>(a, nchunk, s);
}

int upres_norm_blocks(int nx, int ny, int nchunk) {
  return ((nx + RTX - 1) / RTX) * ((ny + RTY - 1) / RTY) * nchunk;
}

template <typename T, typename C> int upres_blocks_per_sm() {
  int blocks = 0;
  constexpr int smem = KS * stage_bytes<T>();
  if (cudaFuncSetAttribute(k_upres_tma<T, C, PG_JACOBI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_upres_tma<T, C, PG_JACOBI>, RNT, smem) != cudaSuccess)
    return 1;
  return blocks > 0 ? blocks : 1;
}

// Bounded-wait self-test: one CTA waits, with `polls` polls, on an mbarrier
// that nothing arrives on -- the situation of a stalled copy in the staged
// kernels -- and, on giving up, sets *err like they do and returns.
__global__ void k_wait_selftest(int* err, int polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  bool ok = false;
  for (int it = 0; it < polls && !ok; ++it) ok = mbar_try_wait(&bar, 0u);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicExch(err, 1);
}

cudaError_t launch_wait_selftest(int* err, int polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, polls);
  return cudaGetLastError();
}

template cudaError_t launch_upres<double, double>(const PgArgs<double, double>&, int, int, cudaStream_t);
template cudaError_t launch_upres<float, float>(const PgArgs<float, float>&, int, int, cudaStream_t);
template cudaError_t launch_upres<__nv_bfloat16, float>(const PgArgs<__nv_bfloat16, float>&, int, int,
                                                        cudaStream_t);
template cudaError_t launch_upres<__half, float>(const PgArgs<__half, float>&, int, int, cudaStream_t);
template int upres_blocks_per_sm<double, double>();
template int upres_blocks_per_sm<float, float>();
template int upres_blocks_per_sm<__nv_bfloat16, float>();
template int upres_blocks_per_sm<__half, float>();

}  // namespace btmg
