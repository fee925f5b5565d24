// k_pg2.cu -- the fused fine PG residual (Eq. Petrov with the anisotropic
// nonlinear dissipation of Sec. 2.6, Eq. ano-k) and the fine PG Jacobi
// sweep (Eq. matrix_full, beta = 3) of k_pg.cu, for FP32 storage and the
// quadratic ConvFEM order, evaluated for TWO directions at a time.
//
// The operator is the same for every direction except for the direction's
// constants (mu, nu, p and the PG limits), so a pair of directions runs
// through the stencil passes as packed FP32x2 values: one fma.rn.f32x2 does
// the work of two FFMA, and the address, integer and control work of every
// pass is shared by both directions.  Each element of a staged field is a
// (direction n, direction n+1) pair; the arithmetic of each lane, and the
// order of every sum, are those of k_pg.cu.
//
// One CTA owns a 32x32 tile and loops over the direction pairs of a chunk.
// The pair's two psi planes arrive by one TMA copy (a 56 x 44 x 2 box) into a
// single staging buffer, which is free again after the first pass, so the
// next pair's copy is issued there and lands during the rest of the passes.
// Passes (D = d1, M = m1, S = s1 of Sec. 2.7 / the Appendix, h = 1):
//   1  A = D_x P, B = D_y P (from the staged planes), Pk = P on the k region
//   2  Px = M_y A / dx, Py = M_x B / dy; derived-field halo
//   3  Tx = M_y Px, Ty = M_y Py; k_x, k_y from M_x T (Eq. ano-k); halo
//   4  U = M_y (k_x pc), M_y k_x, S_y (k_y pc), S_y k_y     (pc = psi - c0)
//   5  per thread and node: the k-free terms S_x M_y pc and M_x S_y pc from
//      pc directly, the x passes of U, D_x = [S_x U0 + k_x S_x M_y pc
//      - pc S_x U1] / dx^2, D_y likewise, r = (b + extra) - (mu Psi_x
//      + nu Psi_y + half (D_x + D_y) + sigma_t psi); residual or Jacobi
//      update of both directions
// Shared arrays of pairs use a chunk swizzle: the pair-chunks (two
// consecutive nodes, both directions: 16 bytes) of a row are stored even
// chunks first, then odd chunks, so that eight threads reading the eight
// chunks 2q (or 2q+1) of eight consecutive quads q touch 128 contiguous
// bytes (no bank conflicts).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "btmg_common.cuh"
#include "tma.cuh"

namespace btmg {
namespace {

constexpr int TX = 32, TY = 32, NT = 256;
constexpr int H6 = TY + 12, W6 = TX + 12;  // psi with its 6-node halo
// staged row: columns x0-8 .. x0+47 (x0+40 .. x0+47 are not used: the
// wider box staggers the banks of staged rows two apart)
constexpr int PS = 56;
constexpr int PLANE = H6 * PS;             // floats of one staged direction plane

// widths (nodes per row) of the pair arrays
constexpr int WA = 40;  // A:  rows y0-6..,  columns x0-4 ..
constexpr int WB = 48;  // B:  rows y0-4..,  columns x0-8 .. (the staged columns)
constexpr int WP = 40;  // Px, Py, Tx, Ty: columns x0-4 ..
constexpr int WK = 36;  // Kx, Ky, Pk, U, V: columns x0-2 ..
constexpr int HA = H6, HB = TY + 8, HPX = TY + 8, HT = TY + 4, HK = TY + 4, HU = TY;

// Row pitch (floats) of each pair array: 2W, plus padding on the arrays
// whose ragged quads (columns 32 and beyond, read by items that span
// several rows) would otherwise put rows two or four apart on the same
// banks; quads 0..7 of a row are 128 contiguous bytes in any case.
template <int W, int RP> struct Lay {
  static_assert(RP >= 2 * W && RP % 4 == 0, "row pitch");
  static constexpr int w = W, rp = RP;
};
using LA = Lay<WA, 2 * WA + 4>;  // A
using LB = Lay<WB, 2 * WB + 8>;  // B
using LP = Lay<WP, 2 * WP + 4>;  // Px, Py
using LT = Lay<WP, 2 * WP + 8>;  // Tx, Ty
using LK = Lay<WK, 2 * WK>;      // Kx, Ky, Pk
using LU = Lay<WK, 2 * WK>;      // U0 .. U3

// float offsets of the arrays (each a multiple of 4 floats)
constexpr int OFF_P = 0;                     // 2 planes, TMA destination
constexpr int OFF_AB = OFF_P + 2 * PLANE;    // A and B, later Tx/Ty, later U0..U3
constexpr int SZ_U = HU * LU::rp;
constexpr int SZ_A = HA * LA::rp, SZ_B = HB * LB::rp, SZ_T = HT * LT::rp;
constexpr int SZ_AB = (SZ_A + SZ_B) > 4 * SZ_U ? (SZ_A + SZ_B) : 4 * SZ_U;
constexpr int OFF_A = OFF_AB, OFF_B = OFF_AB + SZ_A;
constexpr int OFF_TX = OFF_AB, OFF_TY = OFF_AB + SZ_T;
constexpr int OFF_PX = OFF_AB + SZ_AB, OFF_PY = OFF_PX + HPX * LP::rp;
constexpr int OFF_KX = OFF_PY + HPX * LP::rp, OFF_KY = OFF_KX + HK * LK::rp;
constexpr int OFF_PK = OFF_KY + HK * LK::rp;
constexpr int ELEMS = OFF_PK + HK * LK::rp;
static_assert(2 * SZ_T <= SZ_AB, "T arrays inside the A/B region");
static_assert(2 * SZ_U <= 2 * HPX * LP::rp, "U4, U5 inside the Px/Py region");
static_assert(4 * SZ_U <= SZ_AB && SZ_A + SZ_B <= SZ_AB, "A/B region");
static_assert((PLANE * 4) % 128 == 0, "second staged plane 128-byte aligned");
static_assert(OFF_AB % 4 == 0 && OFF_B % 4 == 0 && OFF_TY % 4 == 0 && OFF_PX % 4 == 0 && OFF_PY % 4 == 0 &&
                  OFF_KX % 4 == 0 && OFF_KY % 4 == 0 && OFF_PK % 4 == 0 && SZ_U % 4 == 0,
              "16-byte alignment of the shared arrays");
// two CTAs per SM: 2 x (dynamic + static shared memory + 1 KB reserved) <= 228 KB
static_assert(2 * (ELEMS * 4 + 128 + 1024) <= 228 * 1024, "two CTAs per SM");

// float offset of pair-chunk p (nodes 2p, 2p+1, both directions) of a row of
// an array with layout L
template <class L> __device__ __forceinline__ int chunk(int row, int p) {
  return row * L::rp + (p & 1) * L::w + (p >> 1) * 4;
}
// float offset of node x (lane 0) of a row
template <class L> __device__ __forceinline__ int elem(int row, int x) { return chunk<L>(row, x >> 1) + (x & 1) * 2; }

__device__ __forceinline__ void ld_chunk(const float* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void st_chunk(float* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
// nodes 2p .. 2p+2n-1 of a row (n chunks)
template <class L, int N> __device__ __forceinline__ void ld_run(const float* base, int row, int p, float2 (&o)[2 * N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) ld_chunk(base + chunk<L>(row, p + i), o[2 * i], o[2 * i + 1]);
}
template <class L> __device__ __forceinline__ void st_quad(float* base, int row, int q, const float2 (&o)[4]) {
  st_chunk(base + chunk<L>(row, 2 * q), o[0], o[1]);
  st_chunk(base + chunk<L>(row, 2 * q + 1), o[2], o[3]);
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, exact as a subtraction: fma(b, -1, a)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

// quadratic ConvFEM stencils at offsets -2..2 (h = 1): m1 = (-1,4,24,4,-1)/30,
// s1 = (1,-16,30,-16,1)/12; d1 in difference form on offsets -2,-1,+1,+2
__device__ __forceinline__ float M1(int k) {
  return k == 2 ? 24.0f / 30.0f : ((k == 1 || k == 3) ? 4.0f / 30.0f : -1.0f / 30.0f);
}
__device__ __forceinline__ float S1(int k) {
  return k == 2 ? 30.0f / 12.0f : ((k == 1 || k == 3) ? -16.0f / 12.0f : 1.0f / 12.0f);
}
__device__ __forceinline__ float D1(float p0, float p1, float p3, float p4) {
  return (8.0f / 12.0f) * (p3 - p1) - (1.0f / 12.0f) * (p4 - p0);
}
// 5-tap correlation of NO + 4 consecutive pairs: out[k] = sum_u w_u in[k + u]
template <bool S, int NO> __device__ __forceinline__ void xpass(const float2 (&in)[NO + 4], float2 (&o)[NO]) {
#pragma unroll
  for (int k = 0; k < NO; ++k) {
    float2 acc = mul2(f2(S ? S1(0) : M1(0)), in[k]);
#pragma unroll
    for (int u = 1; u < 5; ++u) acc = fma2(f2(S ? S1(u) : M1(u)), in[k + u], acc);
    o[k] = acc;
  }
}

// Item it of a pass over `rows` row blocks of 8 + E quads: quads 0..7 of a
// row block first (eight consecutive items read one 128-byte run), then the
// E remaining quads of every row block.
template <int E> __device__ __forceinline__ void split_item(int it, int rows, int& rb, int& q) {
  if (it < rows * 8) {
    rb = it >> 3;
    q = it & 7;
  } else {
    const int e = it - rows * 8;
    rb = e / E;
    q = 8 + e % E;
  }
}

// Calls f(r, c) for every cell of an H x W box outside the domain, where box
// cell (r, c) is node (x0 + c - HALO, y0 + r - HALO): the columns left and
// right of the domain over every row, then the rows above and below it
// between those columns (four strips; empty for an interior tile).
// `skip` drops whole strips (bit 0 left, 1 right, 2 top, 3 bottom).
template <int H, int W, int HALO, typename F>
__device__ __forceinline__ void for_outside(int x0, int y0, int nx, int ny, int tid, int copies, F f,
                                            unsigned skip = 0u) {
  const int cl = (skip & 1u) ? 0 : max(0, HALO - x0), ch = (skip & 2u) ? W : min(W, nx - x0 + HALO);
  const int rl = (skip & 4u) ? 0 : max(0, HALO - y0), rh = (skip & 8u) ? H : min(H, ny - y0 + HALO);
  const int mid = ch - cl, wr = W - ch;
  const int nL = H * cl, nR = H * wr, nT = rl * mid, nB = (H - rh) * mid;
  const int tot = nL + nR + nT + nB;
  for (int i = tid; i < copies * tot; i += NT) {
    const int k = i / tot, j = i - k * tot;
    int r, c;
    if (j < nL) {
      r = j / cl, c = j % cl;
    } else if (j < nL + nR) {
      r = (j - nL) / wr, c = ch + (j - nL) % wr;
    } else if (j < nL + nR + nT) {
      r = (j - nL - nR) / mid, c = cl + (j - nL - nR) % mid;
    } else {
      r = rh + (j - nL - nR - nT) / mid, c = cl + (j - nL - nR - nT) % mid;
    }
    f(k, r, c);
  }
}

__global__ void __launch_bounds__(NT, 2) k_pg2(const PgArgs<float, float> a, const int mode,
                                                const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pdl_wait();
  pdl_launch();
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* const P0 = sm + OFF_P;  // staged plane of direction n (tile base: column x0-8, row y0-6)
  float* const P1 = P0 + PLANE;  // direction n+1
  float* const A = sm + OFF_A;
  float* const B = sm + OFF_B;
  float* const Px = sm + OFF_PX;
  float* const Py = sm + OFF_PY;
  float* const Tx = sm + OFF_TX;
  float* const Ty = sm + OFF_TY;
  float* const Kx = sm + OFF_KX;
  float* const Ky = sm + OFF_KY;
  float* const Pk = sm + OFF_PK;
  float* const U0 = sm + OFF_AB;
  float* const U1 = U0 + SZ_U;
  float* const U2 = U1 + SZ_U;
  float* const U3 = U2 + SZ_U;
  float* const U4 = sm + OFF_PX;  // stage 4 on, in place of Px and Py
  float* const U5 = U4 + SZ_U;
  __shared__ double red[NT / 32];
  __shared__ __align__(8) uint64_t bar;

  const int tid = threadIdx.x;
  const int tile = blockIdx.x, chunk_id = a.chunk0 + blockIdx.y;
  const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;
  const bool edge6 = x0 < 6 || y0 < 6 || x0 + TX + 6 > nx || y0 + TY + 6 > ny;
  const bool edge4 = x0 < 4 || y0 < 4 || x0 + TX + 4 > nx || y0 + TY + 4 > ny;

  // stage-5 nodes of this thread: one row, four columns (nx is a multiple
  // of 4, so the four are all inside or all outside in x)
  const int r5 = tid >> 3, c5 = (tid & 7) * 4;
  const int gy5 = y0 + r5, gx5 = x0 + c5;
  const bool in5 = gy5 < ny && gx5 < nx;
  const size_t gi5 = in5 ? (size_t)gy5 * nx + gx5 : 0;
  float sig[4] = {0.f, 0.f, 0.f, 0.f}, bq[4] = {0.f, 0.f, 0.f, 0.f};
  if (in5) {
    const float4 s4 = *reinterpret_cast<const float4*>(a.sigt + gi5);
    const float4 b4 = *reinterpret_cast<const float4*>(a.b + gi5);
    sig[0] = s4.x, sig[1] = s4.y, sig[2] = s4.z, sig[3] = s4.w;
    bq[0] = b4.x, bq[1] = b4.y, bq[2] = b4.z, bq[3] = b4.w;
  }
  double nrm = 0.0;
  float2 acc5[4];  // per lane: sum of p_n r_n (residual) or p_n psi_n (Jacobi)
#pragma unroll
  for (int k = 0; k < 4; ++k) acc5[k] = f2(0.f);

  const int n_begin = chunk_id * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);
  constexpr uint32_t BOX_BYTES = (uint32_t)(2 * PLANE * sizeof(float));
  uint32_t parity = 0;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0 && n_begin < n_end) {
    mbar_expect_tx(&bar, BOX_BYTES);
    tma_load_3d(P0, &tmap, &bar, x0 - 8, y0 - 6, n_begin);
  }
  for (int n = n_begin; n + 1 < n_end; n += 2) {
    const Dir<float> d0 = a.dir[n], d1 = a.dir[n + 1];
    // ---- stage 0: the pair's staged planes ---------------------------------
    {
      const bool got = mbar_wait_bounded(&bar, parity);
      parity ^= 1u;
      if (!__syncthreads_and(got)) {  // copy engine stalled: flag it and leave together
        if (tid == 0) {
          atomicExch(a.err, 1);
          mbar_wait_bounded(&bar, parity ^ 1u);  // the copy still in flight, bounded
        }
        return;
      }
    }
    // out-of-domain cells arrive as 0 (the vacuum incoming halo of Sec. 2.3);
    // the others take the nearest interior node, per direction
    if (edge6) {
      // a strip on an incoming vacuum side is all zero (the copy's fill):
      // skipped whole; the other cells take the nearest interior node
      // unless incoming in the other axis
#pragma unroll
      for (int pl = 0; pl < 2; ++pl) {
        const Dir<float>& dd = pl ? d1 : d0;
        const bool sxp = dd.mu > 0.f, syp = dd.nu > 0.f;
        const unsigned skip = (a.bc.xlo == BC_VACUUM && sxp ? 1u : 0u) | (a.bc.xhi == BC_VACUUM && !sxp ? 2u : 0u) |
                              (a.bc.ylo == BC_VACUUM && syp ? 4u : 0u) | (a.bc.yhi == BC_VACUUM && !syp ? 8u : 0u);
        float* Pp = pl ? P1 : P0;
        for_outside<H6, W6, 6>(
            x0, y0, nx, ny, tid, 1,
            [&](int, int r, int c) {
              const int gx = x0 + c - 6, gy = y0 + r - 6;
              if (!halo_is_zero(a.bc, gx, gy, nx, ny, sxp, syp))
                Pp[r * PS + c + 2] = Pp[(clampi(gy, 0, ny - 1) - y0 + 6) * PS + clampi(gx, 0, nx - 1) - x0 + 8];
            },
            skip);
      }
      __syncthreads();
    }
    // psi at the tile origin, per direction: the product terms use psi - c0
    const float2 c0 = make_float2(P0[6 * PS + 8], P1[6 * PS + 8]);
    float2 adv5[4];  // mu Psi_x + nu Psi_y at this thread's stage-5 nodes
    // ---- stage 1: A = d1_x P, B = d1_y P (difference form), Pk = P ---------
    {
      constexpr int NA = HA * (WA / 4), NB = (HB / 2) * (WB / 4);
#pragma unroll 1
      for (int it = tid; it < NA + NB; it += NT) {
        if (it < NA) {
          int r, q;
          split_item<WA / 4 - 8>(it, HA, r, q);
          const int c = q * 4;
          // A node c is tile column c - 4: inputs at staged columns c + 2 .. c + 9
          float2 o[4], raw[4];
#pragma unroll
          for (int pl = 0; pl < 2; ++pl) {
            const float* Pp = (pl ? P1 : P0) + r * PS + c;
            const float4 q0 = *reinterpret_cast<const float4*>(Pp);
            const float4 q1 = *reinterpret_cast<const float4*>(Pp + 4);
            const float4 q2 = *reinterpret_cast<const float4*>(Pp + 8);
            const float p[8] = {q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y};
            float od[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) od[k] = D1(p[k], p[k + 1], p[k + 3], p[k + 4]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (pl) o[k].y = od[k], raw[k].y = p[k];
              else o[k].x = od[k], raw[k].x = p[k];
            }
          }
          st_quad<LA>(A, r, q, o);
          // Pk: tile rows -2..33, columns -2..33 (A row r = tile row r - 6,
          // the raw inputs p[0..3] are tile columns c - 6 .. c - 3)
          if (r >= 4 && r < 4 + HK && c >= 4 && c <= WK) st_quad<LK>(Pk, r - 4, q - 1, raw);
        } else {
          int rb, q;
          split_item<WB / 4 - 8>(it - NA, HB / 2, rb, q);
          const int r = rb * 2, c = q * 4;  // B rows r, r+1 = tile rows r-4, r-3; staged rows r .. r+5
          float2 o0[4], o1[4];
#pragma unroll
          for (int pl = 0; pl < 2; ++pl) {
            const float* Pp = (pl ? P1 : P0) + r * PS + c;
            float p[6][4];
#pragma unroll
            for (int v = 0; v < 6; ++v) {
              const float4 t = *reinterpret_cast<const float4*>(Pp + v * PS);
              p[v][0] = t.x, p[v][1] = t.y, p[v][2] = t.z, p[v][3] = t.w;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float e0 = D1(p[0][k], p[1][k], p[3][k], p[4][k]);
              const float e1 = D1(p[1][k], p[2][k], p[4][k], p[5][k]);
              if (pl) o0[k].y = e0, o1[k].y = e1;
              else o0[k].x = e0, o1[k].x = e1;
            }
          }
          st_quad<LB>(B, r, q, o0);
          st_quad<LB>(B, r + 1, q, o1);
        }
      }
    }
    __syncthreads();
    // the staged planes are free: request the next pair into them
    if (tid == 0 && n + 2 < n_end) {
      fence_proxy_async();
      mbar_expect_tx(&bar, BOX_BYTES);
      tma_load_3d(P0, &tmap, &bar, x0 - 8, y0 - 6, n + 2);
    }
    // ---- stage 2: Px = m1_y A / dx, Py = m1_x B / dy -----------------------
    {
      const float2 idx = f2(a.inv_dx), idy = f2(a.inv_dy);
      constexpr int NX = (HPX / 2) * (WP / 4), NY = HPX * (WP / 4);
#pragma unroll 1
      for (int it = tid; it < NX + NY; it += NT) {
        if (it < NX) {
          int rb, q;
          split_item<WP / 4 - 8>(it, HPX / 2, rb, q);
          const int r = rb * 2;  // Px rows r, r+1 from A rows r .. r+5
          float2 s0[4], s1[4];
#pragma unroll
          for (int v = 0; v < 6; ++v) {
            float2 p[4];
            ld_run<LA, 2>(A, r + v, 2 * q, p);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (v < 5) s0[k] = v == 0 ? mul2(f2(M1(0)), p[k]) : fma2(f2(M1(v)), p[k], s0[k]);
              if (v > 0) s1[k] = v == 1 ? mul2(f2(M1(0)), p[k]) : fma2(f2(M1(v - 1)), p[k], s1[k]);
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) s0[k] = mul2(s0[k], idx), s1[k] = mul2(s1[k], idx);
          st_quad<LP>(Px, r, q, s0);
          st_quad<LP>(Px, r + 1, q, s1);
        } else {
          int r, q;
          split_item<WP / 4 - 8>(it - NX, HPX, r, q);
          // Py node c = tile column c - 4 needs B nodes c + 2 .. c + 6
          float2 p[8], o[4];
          ld_run<LB, 4>(B, r, 2 * q + 1, p);
          xpass<false>(p, o);
#pragma unroll
          for (int k = 0; k < 4; ++k) o[k] = mul2(o[k], idy);
          st_quad<LP>(Py, r, q, o);
        }
      }
    }
    __syncthreads();
    if (edge4) {  // derived-field halo: nearest interior node
      for_outside<HPX, WP, 4>(x0, y0, nx, ny, tid, 1, [&](int, int r, int c) {
        const int sr = clampi(y0 + r - 4, 0, ny - 1) - y0 + 4, sc = clampi(x0 + c - 4, 0, nx - 1) - x0 + 4;
        *reinterpret_cast<float2*>(Px + elem<LP>(r, c)) = *reinterpret_cast<const float2*>(Px + elem<LP>(sr, sc));
        *reinterpret_cast<float2*>(Py + elem<LP>(r, c)) = *reinterpret_cast<const float2*>(Py + elem<LP>(sr, sc));
      });
      __syncthreads();
    }
    // ---- stage 3a: T = m1_y Psi (rows -2..33), three-row items -------------
    {
      constexpr int NT3 = (HT / 3) * (WP / 4);  // per array
      constexpr int NT3P = (NT3 + 7) / 8 * 8;
#pragma unroll 1
      for (int it = tid; it < 2 * NT3P; it += NT) {
        const bool isx = it < NT3P;
        const int j = isx ? it : it - NT3P;
        if (j >= NT3) continue;
        int rb, q;
        split_item<WP / 4 - 8>(j, HT / 3, rb, q);
        const int r = rb * 3;  // T rows r .. r+2 from Psi rows r .. r+6
        const float* src = isx ? Px : Py;
        float* dst = isx ? Tx : Ty;
        float2 s0[4], s1[4], s2[4];
#pragma unroll
        for (int v = 0; v < 7; ++v) {
          float2 p[4];
          ld_run<LP, 2>(src, r + v, 2 * q, p);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (v < 5) s0[k] = v == 0 ? mul2(f2(M1(0)), p[k]) : fma2(f2(M1(v)), p[k], s0[k]);
            if (v > 0 && v < 6) s1[k] = v == 1 ? mul2(f2(M1(0)), p[k]) : fma2(f2(M1(v - 1)), p[k], s1[k]);
            if (v > 1) s2[k] = v == 2 ? mul2(f2(M1(0)), p[k]) : fma2(f2(M1(v - 2)), p[k], s2[k]);
          }
        }
        st_quad<LT>(dst, r, q, s0);
        st_quad<LT>(dst, r + 1, q, s1);
        st_quad<LT>(dst, r + 2, q, s2);
      }
    }
    __syncthreads();
    // ---- stage 3b: k_x, k_y on tile rows/columns -2..33 (Eq. ano-k) ---------
    {
      const float2 cx = make_float2(a.a_r * d0.mu, a.a_r * d1.mu), cy = make_float2(a.a_r * d0.nu, a.a_r * d1.nu);
      const float amu[2] = {fabsf(d0.mu), fabsf(d1.mu)}, anu[2] = {fabsf(d0.nu), fabsf(d1.nu)};
      const float kxmax[2] = {a.dx * amu[0], a.dx * amu[1]}, kymax[2] = {a.dy * anu[0], a.dy * anu[1]};
      const float2 mu = make_float2(d0.mu, d1.mu), nu = make_float2(d0.nu, d1.nu);
      // K nodes 2p .. 2p + 2NC - 1 of row r (K node c = tile column c - 2):
      // T nodes c .. c + 4 and the Psi node c + 2 of row r + 2; adv = the
      // streaming term mu Psi_x + nu Psi_y of the same nodes
      auto k_nodes = [&](auto nc_tag, int r, int p, auto& adv) {
        constexpr int NC = decltype(nc_tag)::value, NN = 2 * NC;
        float2 tx[NN + 4], ty[NN + 4], pxv[NN], pyv[NN], mx[NN], my[NN];
        ld_run<LT, NC + 2>(Tx, r, p, tx);
        ld_run<LT, NC + 2>(Ty, r, p, ty);
        ld_run<LP, NC>(Px, r + 2, p + 1, pxv);
        ld_run<LP, NC>(Py, r + 2, p + 1, pyv);
        xpass<false>(tx, mx);
        xpass<false>(ty, my);
        float2 kxo[NN], kyo[NN];
#pragma unroll
        for (int k = 0; k < NN; ++k) {
          const float2 Rx = mul2(cx, sub2(mx[k], pxv[k])), Ry = mul2(cy, sub2(my[k], pyv[k]));
          const float rx[2] = {Rx.x, Rx.y}, ry[2] = {Ry.x, Ry.y};
          const float px[2] = {pxv[k].x, pxv[k].y}, py[2] = {pyv[k].x, pyv[k].y};
          float kx[2], ky[2];
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            const float kxa = __fdividef(a.a_kabs * fabsf(rx[l]) * a.dx, a.eps_k + fabsf(px[l]));
            const float kya = __fdividef(a.a_kabs * fabsf(ry[l]) * a.dy, a.eps_k + fabsf(py[l]));
            const float kxs = __fdividef(a.a_ksq * rx[l] * rx[l] * a.dx, a.eps_k + amu[l] * px[l] * px[l]);
            const float kys = __fdividef(a.a_ksq * ry[l] * ry[l] * a.dy, a.eps_k + anu[l] * py[l] * py[l]);
            kx[l] = fminf(fminf(kxmax[l], kxa), kxs);
            ky[l] = fminf(fminf(kymax[l], kya), kys);
          }
          kxo[k] = make_float2(kx[0], kx[1]);
          kyo[k] = make_float2(ky[0], ky[1]);
          adv[k] = fma2(nu, pyv[k], mul2(mu, pxv[k]));
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          st_chunk(Kx + chunk<LK>(r, p + i), kxo[2 * i], kxo[2 * i + 1]);
          st_chunk(Ky + chunk<LK>(r, p + i), kyo[2 * i], kyo[2 * i + 1]);
        }
      };
      // 36 x 36 K nodes: first the stage-5 nodes of this thread (tile row
      // r5, columns c5 .. c5+3: K row r5 + 2, chunks c5/2 + 1, + 2), whose
      // streaming term stays in registers until stage 5; then the other 136
      // chunks as two-node items: K rows 0, 1, 34, 35 (even chunks of a row,
      // then its odd ones) and chunks 0 and 17 of rows 2..33
      static_assert(HK == 36 && WK == 36 && NT == 256, "stage-3b item mapping");
      k_nodes(std::integral_constant<int, 2>{}, r5 + 2, c5 / 2 + 1, adv5);
      if (tid < 136) {
        int r, p;
        if (tid < 72) {
          const int rr = tid / 18, c = tid - rr * 18;
          r = rr < 2 ? rr : rr + 32;
          p = c < 9 ? 2 * c : 2 * (c - 9) + 1;
        } else {
          r = 2 + ((tid - 72) >> 1);
          p = (tid & 1) ? 17 : 0;
        }
        float2 adv_unused[2];
        k_nodes(std::integral_constant<int, 1>{}, r, p, adv_unused);
      }
    }
    __syncthreads();
    if (edge4) {
      for_outside<HK, WK, 2>(x0, y0, nx, ny, tid, 1, [&](int, int r, int c) {
        const int sr = clampi(y0 + r - 2, 0, ny - 1) - y0 + 2, sc = clampi(x0 + c - 2, 0, nx - 1) - x0 + 2;
        *reinterpret_cast<float2*>(Kx + elem<LK>(r, c)) = *reinterpret_cast<const float2*>(Kx + elem<LK>(sr, sc));
        *reinterpret_cast<float2*>(Ky + elem<LK>(r, c)) = *reinterpret_cast<const float2*>(Ky + elem<LK>(sr, sc));
      });
      __syncthreads();
    }
    // ---- stage 4: the y passes of both groups -------------------------------
    //   U0 = m1_y (k_x pc), U1 = m1_y k_x, U4 = m1_y pc,
    //   U2 = s1_y (k_y pc), U3 = s1_y k_y, U5 = s1_y pc
    // on tile rows 0..31, columns -2..33; items of two rows and four nodes
    // (six K and Pk rows in).  U4 and U5 take the place of Px and Py, whose
    // last reads were in stage 3b.
    {
      // two-row items over quads 0..7 of both groups: exactly one per thread
      static_assert((HU / 2) * 8 * 2 == NT && WK / 4 == 9, "stage-4 item mapping");
      {
        const int it = tid;
        const bool xg = it < 128;
        const int j = it & 127;
        const int r = (j >> 3) * 2, q = j & 7;
        const float* K = xg ? Kx : Ky;
        float2 a0[4], a1[4], b0[4], b1[4], e0[4], e1[4];  // rows r and r+1 of the three sums
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          float2 kk[4], pp[4];
          ld_run<LK, 2>(K, r + v, 2 * q, kk);
          ld_run<LK, 2>(Pk, r + v, 2 * q, pp);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 pc = sub2(pp[k], c0);
            const float2 kp = mul2(kk[k], pc);
            if (v < 5) {
              const float2 w = f2(xg ? M1(v) : S1(v));
              a0[k] = v == 0 ? mul2(w, kp) : fma2(w, kp, a0[k]);
              b0[k] = v == 0 ? mul2(w, kk[k]) : fma2(w, kk[k], b0[k]);
              e0[k] = v == 0 ? mul2(w, pc) : fma2(w, pc, e0[k]);
            }
            if (v > 0) {
              const float2 w = f2(xg ? M1(v - 1) : S1(v - 1));
              a1[k] = v == 1 ? mul2(w, kp) : fma2(w, kp, a1[k]);
              b1[k] = v == 1 ? mul2(w, kk[k]) : fma2(w, kk[k], b1[k]);
              e1[k] = v == 1 ? mul2(w, pc) : fma2(w, pc, e1[k]);
            }
          }
        }
        float* dA = xg ? U0 : U2;
        float* dB = xg ? U1 : U3;
        float* dE = xg ? U4 : U5;
        st_quad<LU>(dA, r, q, a0);
        st_quad<LU>(dA, r + 1, q, a1);
        st_quad<LU>(dB, r, q, b0);
        st_quad<LU>(dB, r + 1, q, b1);
        st_quad<LU>(dE, r, q, e0);
        st_quad<LU>(dE, r + 1, q, e1);
      }
      // the ninth quad (nodes 32..35) of every row and group: one node each
      {
        const int it = tid;
        const bool xg = it < 128;
        const int r = (it & 127) >> 2, x = 32 + (it & 3);
        const float* K = xg ? Kx : Ky;
        float2 a = f2(0.f), bsum = f2(0.f), e = f2(0.f);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float2 kk = *reinterpret_cast<const float2*>(K + elem<LK>(r + v, x));
          const float2 pp = *reinterpret_cast<const float2*>(Pk + elem<LK>(r + v, x));
          const float2 pc = sub2(pp, c0);
          const float2 kp = mul2(kk, pc);
          const float2 w = f2(xg ? M1(v) : S1(v));
          a = v == 0 ? mul2(w, kp) : fma2(w, kp, a);
          bsum = v == 0 ? mul2(w, kk) : fma2(w, kk, bsum);
          e = v == 0 ? mul2(w, pc) : fma2(w, pc, e);
        }
        *reinterpret_cast<float2*>((xg ? U0 : U2) + elem<LU>(r, x)) = a;
        *reinterpret_cast<float2*>((xg ? U1 : U3) + elem<LU>(r, x)) = bsum;
        *reinterpret_cast<float2*>((xg ? U4 : U5) + elem<LU>(r, x)) = e;
      }
    }
    __syncthreads();
    // ---- stage 5: x passes and assembly on this thread's four nodes ----------
    {
      // the k-free terms s1_x m1_y pc and m1_x s1_y pc
      float2 u[8], fp[4], gp[4];
      ld_run<LU, 4>(U4, r5, c5 / 2, u);
      xpass<true>(u, fp);
      ld_run<LU, 4>(U5, r5, c5 / 2, u);
      xpass<false>(u, gp);
      float2 fkp[4], fk[4], gkp[4], gk[4];
      ld_run<LU, 4>(U0, r5, c5 / 2, u);
      xpass<true>(u, fkp);
      ld_run<LU, 4>(U1, r5, c5 / 2, u);
      xpass<true>(u, fk);
      ld_run<LU, 4>(U2, r5, c5 / 2, u);
      xpass<false>(u, gkp);
      ld_run<LU, 4>(U3, r5, c5 / 2, u);
      xpass<false>(u, gk);
      // this thread's psi and k (tile row r5, columns c5 .. c5+3)
      float2 praw[4], kxv[4], kyv[4];
      ld_run<LK, 2>(Pk, r5 + 2, c5 / 2 + 1, praw);
      ld_run<LK, 2>(Kx, r5 + 2, c5 / 2 + 1, kxv);
      ld_run<LK, 2>(Ky, r5 + 2, c5 / 2 + 1, kyv);
      const float2 i2x = f2(a.inv_dx2), i2y = f2(a.inv_dy2);
      const float2 half = f2(a.half), w = make_float2(d0.w, d1.w);
      float2 res[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 npc = sub2(c0, praw[k]);  // -(psi - c0)
        const float2 Dx = mul2(fma2(npc, fk[k], fma2(kxv[k], fp[k], fkp[k])), i2x);
        const float2 Dy = mul2(fma2(npc, gk[k], fma2(kyv[k], gp[k], gkp[k])), i2y);
        float2 Ap = fma2(half, add2(Dx, Dy), adv5[k]);
        Ap = fma2(f2(sig[k]), praw[k], Ap);
        res[k] = Ap;
      }
      if (in5) {
        // r = (b + extra) - A psi
        float2 bb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) bb[k] = f2(bq[k]);
        if (a.extra) {
          const float4 e0 = *reinterpret_cast<const float4*>(a.extra + (size_t)n * npix + gi5);
          const float4 e1 = *reinterpret_cast<const float4*>(a.extra + (size_t)(n + 1) * npix + gi5);
          const float ex0[4] = {e0.x, e0.y, e0.z, e0.w}, ex1[4] = {e1.x, e1.y, e1.z, e1.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) bb[k] = add2(bb[k], make_float2(ex0[k], ex1[k]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) res[k] = sub2(bb[k], res[k]);
        if (mode == PG_RESID) {
          *reinterpret_cast<float4*>(a.r_out + (size_t)n * npix + gi5) =
              make_float4(res[0].x, res[1].x, res[2].x, res[3].x);
          *reinterpret_cast<float4*>(a.r_out + (size_t)(n + 1) * npix + gi5) =
              make_float4(res[0].y, res[1].y, res[2].y, res[3].y);
          float n0 = 0.f, n1 = 0.f;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            n0 += res[k].x * res[k].x;
            n1 += res[k].y * res[k].y;
            acc5[k] = fma2(w, res[k], acc5[k]);
          }
          nrm += (double)d0.w * (double)n0 + (double)d1.w * (double)n1;
        } else {
          float pn[2][4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float dd0 = a.beta * (d0.ax + d0.ay + sig[k]), dd1 = a.beta * (d1.ax + d1.ay + sig[k]);
            pn[0][k] = praw[k].x + __fdividef(res[k].x, dd0);
            pn[1][k] = praw[k].y + __fdividef(res[k].y, dd1);
            acc5[k] = fma2(w, make_float2(pn[0][k], pn[1][k]), acc5[k]);
          }
          *reinterpret_cast<float4*>(a.psi_out + (size_t)n * npix + gi5) =
              make_float4(pn[0][0], pn[0][1], pn[0][2], pn[0][3]);
          *reinterpret_cast<float4*>(a.psi_out + (size_t)(n + 1) * npix + gi5) =
              make_float4(pn[1][0], pn[1][1], pn[1][2], pn[1][3]);
        }
      }
    }
    // the next pair's first barrier orders these reads of U, Pk, Px, Py and
    // K before that pair's first pass rewrites them
  }
  float phi4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) phi4[k] = acc5[k].x + acc5[k].y;
  if (mode == PG_JACOBI) {
    if (in5)
      *reinterpret_cast<float4*>(a.phi_part + (size_t)chunk_id * npix + gi5) =
          make_float4(phi4[0], phi4[1], phi4[2], phi4[3]);
  } else {
    if (a.rho_part && in5)
      *reinterpret_cast<float4*>(a.rho_part + (size_t)chunk_id * npix + gi5) =
          make_float4(phi4[0], phi4[1], phi4[2], phi4[3]);
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) red[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      a.norm_part[(size_t)chunk_id * gridDim.x + blockIdx.x] = s * (double)a.dxdy;
    }
  }
}

}  // namespace

// The paired kernel takes FP32 storage with rows of a multiple of 4 nodes
// (the TMA row stride and the 16-byte stores of stage 5) and an even number
// of directions per chunk; false means "use k_pg".
bool pg2_applies(const PgArgs<float, float>& a) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) % 16) == 0; };
  return a.order == 2 && a.nx % 4 == 0 && a.dpc % 2 == 0 && al(a.psi) && al(a.sigt) && al(a.b) && al(a.extra) &&
         al(a.r_out) && al(a.psi_out) && al(a.phi_part) && al(a.rho_part) && tmap_encoder() != nullptr;
}

int pg2_blocks_per_sm() {
  constexpr size_t smem = (size_t)ELEMS * sizeof(float);
  if (cudaFuncSetAttribute(k_pg2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
  int blocks = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_pg2, NT, smem) != cudaSuccess) return 1;
  return blocks < 1 ? 1 : blocks;
}

cudaError_t launch_pg2(const PgArgs<float, float>& a, int mode, int nchunk, cudaStream_t s) {
  constexpr size_t smem = (size_t)ELEMS * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_pg2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  if (!encode_tmap_3d(&tm, a.psi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), a.nx, a.ny, a.nd, PS, H6, 2))
    return cudaErrorInvalidValue;
  const int tiles_y = (a.ny + TY - 1) / TY;
  dim3 grid(a.tiles_x * tiles_y, nchunk);
  return launch_pdl(k_pg2, grid, dim3(NT), smem, s, a, mode, tm);
}

}  // namespace btmg
