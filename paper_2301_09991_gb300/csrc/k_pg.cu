// k_pg.cu -- fused fine-level Petrov-Galerkin residual (Eq. Petrov with the
// anisotropic nonlinear dissipation of Sec. 2.6) and fine PG Jacobi sweep
// (Eq. matrix_full, beta = 3).
//
// One CTA owns a 32x32 tile of nodes and loops over a chunk of directions.
// For every direction the tile plus a 6-node halo of psi is staged in shared
// memory (halo rule of Sec. 2.3 applied on load), and the whole operator is
// evaluated from shared memory with the quadratic ConvFEM filters written as
// separable 1D passes (every 5x5 filter of the Appendix is a tensor product
// of m1 = (-1,4,24,4,-1)/30, d1 = (1,-8,0,8,-1)/12 and
// s1 = (1,-16,30,-16,1)/12):
//   Psi_x = m1_y d1_x psi / dx,            Psi_y = m1_x d1_y psi / dy
//   R_x = a_r mu (m1_x m1_y - I) Psi_x,    R_y likewise        (Sec. 2.6)
//   k_x = min(dx|mu|, a_kabs|R_x|dx/(eps+|Psi_x|), a_ksq R_x^2 dx/(eps+|mu|Psi_x^2))
//   D_x = [s1_x m1_y (k_x psi) + k_x s1_x m1_y psi - psi s1_x m1_y k_x] / dx^2
//   r   = b - (mu Psi_x + nu Psi_y + half (D_x + D_y) + sigma_t psi)
// Dependency depth: D needs k on +-2, k needs Psi_x on +-2, Psi_x needs psi
// on +-2, hence the 6-node halo.  Derived fields (Psi_x, Psi_y, k_x, k_y)
// take the value of the nearest interior node outside the domain.
//
// Every pass is register blocked with a compile-time work mapping: a thread
// produces 4 consecutive x outputs (x passes, two 16-byte shared loads) or a
// 4-wide block of 2 or 4 rows (y passes).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "btmg_common.cuh"
#include "tma.cuh"

namespace btmg {
namespace {

constexpr int TX = 32, TY = 32, NT = 256;
constexpr int W6 = TX + 12, H6 = TY + 12;  // 44
constexpr int W4 = TX + 8, H4 = TY + 8;    // 40
constexpr int W2 = TX + 4, H2 = TY + 4;    // 36

// ConvFEM 1D stencils (offsets -2..2), h = 1, of order ORD (Sec. 2.7 and the
// Appendix): quadratic m1 = (-1,4,24,4,-1)/30, d1 = (1,-8,0,8,-1)/12,
// s1 = (1,-16,30,-16,1)/12; linear m1 = (1,4,1)/6, d1 = (-1,0,1)/2,
// s1 = (-1,2,-1), written with zero outer taps (the 3x3 filters are
// tensor products of them).
template <typename C, int ORD> __device__ __forceinline__ C M1(int k) {
  if (ORD == 1) return k == 2 ? C(4.0 / 6.0) : ((k == 1 || k == 3) ? C(1.0 / 6.0) : C(0));
  return k == 2 ? C(24.0 / 30.0) : ((k == 1 || k == 3) ? C(4.0 / 30.0) : C(-1.0 / 30.0));
}
template <typename C, int ORD> __device__ __forceinline__ C S1(int k) {
  if (ORD == 1) return k == 2 ? C(2.0) : ((k == 1 || k == 3) ? C(-1.0) : C(0));
  return k == 2 ? C(30.0 / 12.0) : ((k == 1 || k == 3) ? C(-16.0 / 12.0) : C(1.0 / 12.0));
}
// d1 in difference form on the values at offsets -2, -1, +1, +2
template <typename C, int ORD> __device__ __forceinline__ C D1(C p0, C p1, C p3, C p4) {
  if (ORD == 1) return C(0.5) * (p3 - p1);
  return C(8.0 / 12.0) * (p3 - p1) - C(1.0 / 12.0) * (p4 - p0);
}

// 4 consecutive elements from / to 16-byte aligned shared memory
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&o)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&o)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
}
// 4 consecutive elements starting on an 8-byte boundary (two pairs)
__device__ __forceinline__ void ld2x2(const float* p, float (&o)[4]) {
  const float2 a = *reinterpret_cast<const float2*>(p), b = *reinterpret_cast<const float2*>(p + 2);
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}
__device__ __forceinline__ void ld2x2(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}
// 8 consecutive elements (two aligned quads)
template <typename C> __device__ __forceinline__ void ld8(const C* p, C (&o)[8]) {
  C a[4], b[4];
  ld4(p, a);
  ld4(p + 4, b);
#pragma unroll
  for (int k = 0; k < 4; ++k) o[k] = a[k], o[k + 4] = b[k];
}

template <typename C> __device__ __forceinline__ C cmin(C a, C b) { return a < b ? a : b; }

// Item it of a pass over `rows` row blocks of 8 + E quads: the quads 0..7 of
// a row block first (eight consecutive items = the eight threads of one
// 128-bit access phase read one 32-element row segment, no bank
// conflicts), then the E remaining quads of every row block.
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
// FP32: the fast division intrinsic (2 ulp; the PG coefficients and the
// Jacobi step tolerate it); FP64: exact division.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float cabs_(float v) { return fabsf(v); }
__device__ __forceinline__ double cabs_(double v) { return fabs(v); }

// Shared-memory layout in elements; every array starts on a 4-element
// boundary and every row stride (44, 40, 36) is a multiple of 4.
//   P   two H6 x PS tiles (double buffer), origin (-6,-8): psi   stages 0-5
//       (the pointer P used below is offset by 2: P[r * PS + c] is (r-6, c-6))
//   A   H6 x W4, origin (-6,-4): d1_x P                   stages 1-2
//   B   H4 x PS, origin (-4,-8): d1_y P (the staged tile's 16-byte aligned
//       column quads; columns -8, -7, 38, 39 are never read)  stages 1-2
//   Px, Py  H4 x W4, origin (-4,-4)                       stages 2-5
//   Kx, Ky  H2 x W2, origin (-2,-2)                       stages 3-5
//   Tx, Ty  H2 x W4, origin (-2,-4): m1_y Psi  (in the dead A/B region)  stage 3
//   V1..V3  TY x W2, origin (0,-2): s1_y pass  (in the dead A/B region)  stages 4-5
//   U1, U2, W1  TY x W2, origin (0,-2): m1_y pass (after Ky)          stages 4-5
constexpr int PS = 48;                 // row stride of the staged psi tile
constexpr int PBUF = H6 * PS;          // one staged tile: rows -6.., cols -8..
constexpr int OFF_P = 0;               // two tiles (double buffer)
constexpr int OFF_A = OFF_P + 2 * PBUF;
constexpr int OFF_B = OFF_A + H6 * W4;
constexpr int OFF_PX = OFF_B + H4 * PS;
constexpr int OFF_PY = OFF_PX + H4 * W4;
constexpr int OFF_KX = OFF_PY + H4 * W4;
constexpr int OFF_KY = OFF_KX + H2 * W2;
constexpr int S4N = TY * W2;
constexpr int OFF_U = OFF_KY + H2 * W2;
constexpr int OFF_TX = OFF_A;
constexpr int OFF_TY = OFF_A + H2 * W4;
constexpr int OFF_V = OFF_A;
// Aligned copy of the staged tile over the k region (rows 4..39, columns
// -2..33 of the tile: the origin of Kx/Ky), written by the x-derivative pass
// from its aligned loads and read by the k-Diff y passes with 128-bit loads
// (the staged tile itself is 8-byte aligned there: conflicting pair loads).
constexpr int OFF_PK = OFF_U + 3 * S4N;
constexpr int PG_ELEMS = OFF_PK + H2 * W2;
static_assert(OFF_TY + H2 * W4 <= OFF_PX, "T arrays must stay inside the dead A/B region");
static_assert(OFF_V + 3 * S4N <= OFF_PX, "V arrays must stay inside the dead A/B region");
static_assert((PBUF * 4) % 128 == 0, "TMA destinations must be 128-byte aligned");
static_assert(OFF_A % 4 == 0 && OFF_B % 4 == 0 && OFF_PX % 4 == 0 && OFF_PY % 4 == 0 && OFF_KX % 4 == 0 &&
                  OFF_KY % 4 == 0 && OFF_U % 4 == 0 && OFF_TY % 4 == 0 && S4N % 4 == 0,
              "16-byte alignment of the shared arrays");

template <typename T, typename C, int MODE, bool PGON, bool TMA, int ORD>
__global__ void __launch_bounds__(NT, sizeof(C) == 4 ? 3 : 1)
    k_pg(const PgArgs<T, C> a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pdl_wait();
  pdl_launch();
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* P = sm + OFF_P + 2;  // current staged tile (+2: origin -6 in x)
  C* A = sm + OFF_A;
  C* B = sm + OFF_B;
  C* Px = sm + OFF_PX;
  C* Py = sm + OFF_PY;
  C* Kx = sm + OFF_KX;
  C* Ky = sm + OFF_KY;
  C* Tx = sm + OFF_TX;
  C* Ty = sm + OFF_TY;
  C* Pk = sm + OFF_PK;
  C* U1 = sm + OFF_U;
  C* U2 = U1 + S4N;
  C* W1 = U2 + S4N;
  C* V1 = sm + OFF_V;
  C* V2 = V1 + S4N;
  C* V3 = V2 + S4N;
  __shared__ double red[NT / 32];
  __shared__ __align__(8) uint64_t bars[2];

  const int tid = threadIdx.x;
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;
  // tiles whose 4-halo leaves the domain need the derived-field fill passes
  const bool edge = x0 < 4 || y0 < 4 || x0 + TX + 4 > nx || y0 + TY + 4 > ny;

  double nrm = 0.0;
  C phi_acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) phi_acc[k] = C(0);
  // stage-5 mapping: one row, four consecutive columns
  const int r5 = tid >> 3, c5 = (tid & 7) * 4;

  const int n_begin = chunk * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);
  constexpr uint32_t TILE_BYTES = (uint32_t)(PBUF * sizeof(C));
  uint32_t phase = 0;  // bit b: parity of buffer b's next completion
  if (TMA) {
    if (tid == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0 && n_begin < n_end) {
      mbar_expect_tx(&bars[0], TILE_BYTES);
      tma_load_3d(sm + OFF_P, &tmap, &bars[0], x0 - 8, y0 - 6, n_begin);
    }
  }
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    const T* psin = a.psi + (size_t)n * npix;
    // ---- stage 0: psi with halo -------------------------------------------
    if (TMA) {
      // The tile of direction n was requested one direction earlier; request
      // the next one into the other buffer (released by the barrier that
      // ended the previous direction), then wait for this one.
      const int b = (n - n_begin) & 1;
      if (tid == 0 && n + 1 < n_end) {
        fence_proxy_async();
        mbar_expect_tx(&bars[b ^ 1], TILE_BYTES);
        tma_load_3d(sm + OFF_P + (b ^ 1) * PBUF, &tmap, &bars[b ^ 1], x0 - 8, y0 - 6, n + 1);
      }
      const bool got = mbar_wait_bounded(&bars[b], (phase >> b) & 1u);
      phase ^= 1u << b;
      if (!__syncthreads_and(got)) {  // copy engine stalled: flag it and leave together
        if (tid == 0) {
          atomicExch(a.err, 1);
          if (n + 1 < n_end) mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u);
        }
        return;
      }
      P = sm + OFF_P + b * PBUF + 2;
      // out-of-domain cells arrive as 0 (the vacuum incoming halo); the
      // others take the nearest interior node (boundary tiles only)
      if (x0 < 6 || y0 < 6 || x0 + TX + 6 > nx || y0 + TY + 6 > ny) {
        for (int i = tid; i < H6 * W6; i += NT) {
          const int r = i / W6, c = i % W6;
          const int gx = x0 + c - 6, gy = y0 + r - 6;
          if ((gx < 0 || gx >= nx || gy < 0 || gy >= ny) && !halo_is_zero(a.bc, gx, gy, nx, ny, sxp, syp))
            P[r * PS + c] = P[(clampi(gy, 0, ny - 1) - y0 + 6) * PS + clampi(gx, 0, nx - 1) - x0 + 6];
        }
        __syncthreads();
      }
    } else {
#pragma unroll 2
      for (int i = tid; i < H6 * PS; i += NT) {  // the box's 48 columns, like the TMA copy
        const int gx = x0 + (i % PS) - 8, gy = y0 + (i / PS) - 6;
        C v;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny)
          v = Conv<T>::ld(psin + (size_t)gy * nx + gx);
        else if (halo_is_zero(a.bc, gx, gy, nx, ny, sxp, syp))
          v = C(0);
        else
          v = Conv<T>::ld(psin + (size_t)clampi(gy, 0, ny - 1) * nx + clampi(gx, 0, nx - 1));
        P[i - 2] = v;  // P - 2 is the tile base
      }
      __syncthreads();
    }
    // Every derivative term is unchanged by a constant shift of psi (all
    // those filters sum to zero).  The derivative passes are evaluated in
    // difference form; the product terms of stages 4 and 5 use psi - c0
    // (c0 = psi at the tile origin), so they round relative to the local
    // variation of psi, not to its magnitude.
    const C c0 = PGON ? P[6 * PS + 6] : C(0);
    if constexpr (PGON) {
      // ---- stage 1: derivative passes in difference form --------------------
      // A = d1_x P: items (row, quad); B = d1_y P: items (row pair, quad)
      {
        constexpr int NA = H6 * (W4 / 4), NB = (H4 / 2) * (PS / 4);
#pragma unroll
        for (int it = tid; it < NA + NB; it += NT) {
          if (it < NA) {
            int r, q;
            split_item<W4 / 4 - 8>(it, H6, r, q);
            const int c = q * 4;
            // inputs at (r-6, c-6 .. c+1) = tile columns c+2 .. c+9: three
            // aligned quads starting at tile column c (P - 2 is the tile base)
            C q0[4], q1[4], q2[4], o[4];
            ld4(P - 2 + r * PS + c, q0);
            ld4(P - 2 + r * PS + c + 4, q1);
            ld4(P - 2 + r * PS + c + 8, q2);
            const C p[8] = {q0[2], q0[3], q1[0], q1[1], q1[2], q1[3], q2[0], q2[1]};
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = D1<C, ORD>(p[k], p[k + 1], p[k + 3], p[k + 4]);
            st4(A + r * W4 + c, o);
            if (r >= 4 && r < 4 + H2 && c >= 4 && c <= W2) {  // tile rows -2..33, columns -2..33
              const C pk[4] = {q0[2], q0[3], q1[0], q1[1]};
              st4(Pk + (r - 4) * W2 + (c - 4), pk);
            }
          } else {
            int rb, q;
            split_item<PS / 4 - 8>(it - NA, H4 / 2, rb, q);
            const int r = rb * 2, c = q * 4;  // B column c = tile column c - 8
            C p[6][4];
#pragma unroll
            for (int v = 0; v < 6; ++v) ld4(P - 2 + (r + v) * PS + c, p[v]);
            C o0[4], o1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              o0[k] = D1<C, ORD>(p[0][k], p[1][k], p[3][k], p[4][k]);
              o1[k] = D1<C, ORD>(p[1][k], p[2][k], p[4][k], p[5][k]);
            }
            st4(B + r * PS + c, o0);
            st4(B + (r + 1) * PS + c, o1);
          }
        }
      }
      __syncthreads();
      // ---- stage 2: mass passes: Psi_x = m1_y A / dx, Psi_y = m1_x B / dy ---
      {
        constexpr int NX = (H4 / 2) * (W4 / 4), NY = H4 * (W4 / 4);
#pragma unroll
        for (int it = tid; it < NX + NY; it += NT) {
          if (it < NX) {
            int rb, q;
            split_item<W4 / 4 - 8>(it, H4 / 2, rb, q);
            const int r = rb * 2, c = q * 4;
            C p[6][4];
#pragma unroll
            for (int v = 0; v < 6; ++v) ld4(A + (r + v) * W4 + c, p[v]);
            C o0[4], o1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              C s0 = C(0), s1 = C(0);
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                s0 += M1<C, ORD>(v) * p[v][k];
                s1 += M1<C, ORD>(v) * p[v + 1][k];
              }
              o0[k] = s0 * a.inv_dx;
              o1[k] = s1 * a.inv_dx;
            }
            st4(Px + r * W4 + c, o0);
            st4(Px + (r + 1) * W4 + c, o1);
          } else {
            int r, q;
            split_item<W4 / 4 - 8>(it - NX, H4, r, q);
            const int c = q * 4;
            // inputs at tile columns c - 6 .. c + 1 = B columns c + 2 .. c + 9:
            // three aligned quads starting at B column c
            C b0[4], b1[4], b2[4], o[4];
            ld4(B + r * PS + c, b0);
            ld4(B + r * PS + c + 4, b1);
            ld4(B + r * PS + c + 8, b2);
            const C p[8] = {b0[2], b0[3], b1[0], b1[1], b1[2], b1[3], b2[0], b2[1]};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              C s = C(0);
#pragma unroll
              for (int u = 0; u < 5; ++u) s += M1<C, ORD>(u) * p[k + u];
              o[k] = s * a.inv_dy;
            }
            st4(Py + r * W4 + c, o);
          }
        }
      }
      __syncthreads();
      if (edge) {  // derived-field halo: nearest interior node
        for (int i = tid; i < H4 * W4; i += NT) {
          const int gx = x0 + (i % W4) - 4, gy = y0 + (i / W4) - 4;
          if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
            const int j = (clampi(gy, 0, ny - 1) - y0 + 4) * W4 + (clampi(gx, 0, nx - 1) - x0 + 4);
            Px[i] = Px[j];
            Py[i] = Py[j];
          }
        }
        __syncthreads();
      }
      // ---- stage 3: T = m1_y Psi (4-row blocks), then k on the 2-halo -------
      {
        constexpr int NT3 = (H2 / 4) * (W4 / 4);  // per array
        constexpr int NT3P = (NT3 + 7) / 8 * 8;    // the second array starts on a phase
#pragma unroll
        for (int it = tid; it < 2 * NT3P; it += NT) {
          const bool isx = it < NT3P;
          const int j = isx ? it : it - NT3P;
          if (j >= NT3) continue;
          int rb, q;
          split_item<W4 / 4 - 8>(j, H2 / 4, rb, q);
          const int r = rb * 4, c = q * 4;
          const C* src = isx ? Px : Py;
          C* dst = isx ? Tx : Ty;
          C p[8][4];
#pragma unroll
          for (int v = 0; v < 8; ++v) ld4(src + (r + v) * W4 + c, p[v]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            C o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              C s = C(0);
#pragma unroll
              for (int v = 0; v < 5; ++v) s += M1<C, ORD>(v) * p[q + v][k];
              o[k] = s;
            }
            st4(dst + (r + q) * W4 + c, o);
          }
        }
      }
      __syncthreads();
      {
        const C amu = cabs_(dr.mu), anu = cabs_(dr.nu);
        const C kxmax = a.dx * amu, kymax = a.dy * anu;
        const C cx = a.a_r * dr.mu, cy = a.a_r * dr.nu;
        constexpr int NK = H2 * (W2 / 4);
#pragma unroll
        for (int it = tid; it < NK; it += NT) {
          int r, q;
          split_item<W2 / 4 - 8>(it, H2, r, q);
          const int c = q * 4;
          C tx[8], ty[8];
          ld8(Tx + r * W4 + c, tx);
          ld8(Ty + r * W4 + c, ty);
          C kxo[4], kyo[4], pxv[4], pyv[4];
          ld2x2(Px + (r + 2) * W4 + c + 2, pxv);
          ld2x2(Py + (r + 2) * W4 + c + 2, pyv);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            C mx = C(0), my = C(0);
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              mx += M1<C, ORD>(u) * tx[k + u];
              my += M1<C, ORD>(u) * ty[k + u];
            }
            const C pxc = pxv[k], pyc = pyv[k];
            const C Rx = cx * (mx - pxc), Ry = cy * (my - pyc);
            const C kxa = fdiv(a.a_kabs * cabs_(Rx) * a.dx, a.eps_k + cabs_(pxc));
            const C kya = fdiv(a.a_kabs * cabs_(Ry) * a.dy, a.eps_k + cabs_(pyc));
            const C kxs = fdiv(a.a_ksq * Rx * Rx * a.dx, a.eps_k + amu * pxc * pxc);
            const C kys = fdiv(a.a_ksq * Ry * Ry * a.dy, a.eps_k + anu * pyc * pyc);
            kxo[k] = cmin(cmin(kxmax, kxa), kxs);
            kyo[k] = cmin(cmin(kymax, kya), kys);
          }
          st4(Kx + r * W2 + c, kxo);
          st4(Ky + r * W2 + c, kyo);
        }
      }
      __syncthreads();
      if (edge) {
        for (int i = tid; i < H2 * W2; i += NT) {
          const int gx = x0 + (i % W2) - 2, gy = y0 + (i / W2) - 2;
          if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
            const int j = (clampi(gy, 0, ny - 1) - y0 + 2) * W2 + (clampi(gx, 0, nx - 1) - x0 + 2);
            Kx[i] = Kx[j];
            Ky[i] = Ky[j];
          }
        }
        __syncthreads();
      }
      // ---- stage 4: y passes of the k-Diff terms (2-row blocks) -------------
      //   x group: u1 = m1_y (k_x P), u2 = m1_y k_x, w1 = m1_y P
      //   y group: v1 = s1_y (k_y P), v2 = s1_y k_y, v3 = s1_y P
      // Items (group, row pair, quad): the eight quads 0..7 of a row pair go
      // to the eight threads of one 128-bit access phase, which then read
      // one 32-element row segment (no bank conflicts); the ninth quad
      // (columns 32..35) of every row pair is a second pass of one warp.
      {
        static_assert(W2 == 36 && TY == 32 && NT == 256, "stage-4 item mapping");
        auto s4item = [&](const bool xg, const int r, const int c) {
          const C* K = xg ? Kx : Ky;
          // the 6 input rows stream through: row v adds to output row 0 with
          // tap v and to output row 1 with tap v - 1 (same sums, same order)
          C o[2][3][4];
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
              for (int k = 0; k < 4; ++k) o[q][m][k] = C(0);
#pragma unroll
          for (int v = 0; v < 6; ++v) {
            C kk[4], pp[4], pk[4], kp[4];
            ld4(K + (r + v) * W2 + c, kk);
            ld4(Pk + (r + v) * W2 + c, pp);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              pk[k] = pp[k] - c0;
              kp[k] = kk[k] * pk[k];  // shared by both output rows
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int tap = v - q;
              if (tap < 0 || tap > 4) continue;
              const C w = xg ? M1<C, ORD>(tap) : S1<C, ORD>(tap);
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                o[q][0][k] += w * kp[k];
                o[q][1][k] += w * kk[k];
                o[q][2][k] += w * pk[k];
              }
            }
          }
          C* d0 = xg ? U1 : V1;
          C* d1 = xg ? U2 : V2;
          C* d2 = xg ? W1 : V3;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            st4(d0 + (r + q) * W2 + c, o[q][0]);
            st4(d1 + (r + q) * W2 + c, o[q][1]);
            st4(d2 + (r + q) * W2 + c, o[q][2]);
          }
        };
        s4item(tid < 128, ((tid & 127) >> 3) * 2, (tid & 7) * 4);
        if (tid < 32) s4item(tid < 16, (tid & 15) * 2, 32);
      }
      __syncthreads();
    }  // PGON
    // ---- stage 5: assemble r on the tile (one row, four columns) -----------
    {
      const int ry = r5, rx = c5;
      const int gy = y0 + ry;
      C fkp[4], fp[4], fk[4], gkp[4], gp[4], gk[4];
      if constexpr (PGON) {
        // x group, then y group: three 8-wide rows live at a time
        auto xpass = [&](const C* src, const bool sx, C (&o)[4]) {
          C v[8];
          ld8(src + ry * W2 + rx, v);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            C acc = C(0);
#pragma unroll
            for (int u = 0; u < 5; ++u) acc += (sx ? S1<C, ORD>(u) : M1<C, ORD>(u)) * v[k + u];
            o[k] = acc;
          }
        };
        xpass(U1, true, fkp);
        xpass(U2, true, fk);
        xpass(W1, true, fp);
        xpass(V1, false, gkp);
        xpass(V2, false, gk);
        xpass(V3, false, gp);
      }
      C pcv[4], pxv[4], pyv[4], kxv[4], kyv[4];
      ld4(P + (ry + 6) * PS + rx + 6, pcv);  // box column rx + 8: 16-byte aligned
#pragma unroll
      for (int k = 0; k < 4; ++k) pcv[k] -= c0;  // psi - c0
      if constexpr (PGON) {
        ld4(Px + (ry + 4) * W4 + rx + 4, pxv);
        ld4(Py + (ry + 4) * W4 + rx + 4, pyv);
        ld2x2(Kx + (ry + 2) * W2 + rx + 2, kxv);
        ld2x2(Ky + (ry + 2) * W2 + rx + 2, kyv);
      }
      C nrm_dir = C(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int gx = x0 + rx + k;
        if (gx >= nx || gy >= ny) continue;
        const C pc = pcv[k];
        const size_t gi = (size_t)gy * nx + gx;
        const C psi_c = Conv<T>::ld(psin + gi);  // unshifted psi of this node
        const C sig = a.sigt[gi];
        C Apsi;
        if constexpr (PGON) {
          const C Dx = (fkp[k] + kxv[k] * fp[k] - pc * fk[k]) * a.inv_dx2;
          const C Dy = (gkp[k] + kyv[k] * gp[k] - pc * gk[k]) * a.inv_dy2;
          Apsi = dr.mu * pxv[k] + dr.nu * pyv[k] + a.half * (Dx + Dy) + sig * psi_c;
        } else {
          // upwind filters of Sec. 2.4 (one-sided by the signs of mu and nu)
          const C ux = sxp ? (pc - P[(ry + 6) * PS + rx + k + 5]) : (P[(ry + 6) * PS + rx + k + 7] - pc);
          const C uy = syp ? (pc - P[(ry + 5) * PS + rx + k + 6]) : (P[(ry + 7) * PS + rx + k + 6] - pc);
          Apsi = dr.mu * ux * a.inv_dx + dr.nu * uy * a.inv_dy + sig * psi_c;
        }
        const C r = a.b[gi] + (a.extra ? a.extra[(size_t)n * npix + gi] : C(0)) - Apsi;
        if (MODE == PG_RESID) {
          a.r_out[(size_t)n * npix + gi] = r;
          nrm_dir += r * r;
          phi_acc[k] += dr.w * r;  // residual moment (used when rho_part is set)
        } else {
          const C d = a.beta * (dr.ax + dr.ay + sig);
          const C pn = psi_c + fdiv(r, d);
          Conv<T>::st(a.psi_out + (size_t)n * npix + gi, pn);
          phi_acc[k] += dr.w * stored<T, C>(pn);
        }
      }
      // one FP64 accumulation per direction (the FP64 pipe is narrow)
      if (MODE == PG_RESID) nrm += (double)dr.w * (double)nrm_dir;
    }
    __syncthreads();
  }
  if (MODE == PG_JACOBI) {
    C* ph = a.phi_part + (size_t)chunk * npix;
    const int gy = y0 + r5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int gx = x0 + c5 + k;
      if (gx < nx && gy < ny) ph[(size_t)gy * nx + gx] = phi_acc[k];
    }
  } else {
    if (a.rho_part) {
      C* rh = a.rho_part + (size_t)chunk * npix;
      const int gy = y0 + r5;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int gx = x0 + c5 + k;
        if (gx < nx && gy < ny) rh[(size_t)gy * nx + gx] = phi_acc[k];
      }
    }
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) red[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      a.norm_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s * (double)a.dxdy;
    }
  }
}

template <typename C, bool PGON> constexpr size_t smem_bytes() {
  // the upwind variant only needs the staged psi tiles
  return (PGON ? (size_t)PG_ELEMS : (size_t)(2 * PBUF)) * sizeof(C);
}

// 3D tensor map over psi (x, y, direction) with a 48 x 44 x 1 box; the box
// starts at x0 - 8, a multiple of 8 elements (the innermost coordinate of a
// TMA copy must be 16-byte aligned).  Used when psi is stored in the compute
// type, its base is 16-byte aligned and a row is a multiple of 16 bytes.
template <typename T, typename C> bool make_tmap(CUtensorMap* m, const PgArgs<T, C>& a) {
  if (sizeof(T) != sizeof(C)) return false;
  const size_t es = sizeof(T);
  return encode_tmap_3d(m, a.psi, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, es,
                        a.nx, a.ny, a.nd, PS, H6);
}

template <typename T, typename C, int MODE, bool PGON, bool TMA, int ORD>
cudaError_t launch_variant(const PgArgs<T, C>& a, const CUtensorMap& tm, int nchunk, cudaStream_t s) {
  constexpr size_t smem = smem_bytes<C, PGON>();
  static bool attr_set = false;  // per instantiation, once per process
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(k_pg<T, C, MODE, PGON, TMA, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tiles_y = (a.ny + TY - 1) / TY;
  dim3 grid(a.tiles_x * tiles_y, nchunk);
  return launch_pdl(k_pg<T, C, MODE, PGON, TMA, ORD>, grid, dim3(NT), smem, s, a, tm);
}

template <typename T, typename C, int MODE, bool PGON, int ORD>
cudaError_t launch_order(const PgArgs<T, C>& a, int nchunk, cudaStream_t s) {
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  if constexpr (sizeof(T) == sizeof(C)) {
    if (make_tmap(&tm, a)) return launch_variant<T, C, MODE, PGON, true, ORD>(a, tm, nchunk, s);
  }
  return launch_variant<T, C, MODE, PGON, false, ORD>(a, tm, nchunk, s);
}

// the linear order is built for FP64 and FP32 storage
template <typename T, typename C, int MODE, bool PGON>
cudaError_t launch_mode(const PgArgs<T, C>& a, int nchunk, cudaStream_t s) {
  if constexpr (sizeof(T) == sizeof(C)) {
    if (a.order == 1) return launch_order<T, C, MODE, PGON, 1>(a, nchunk, s);
  }
  if (a.order != 2) return cudaErrorNotSupported;
  return launch_order<T, C, MODE, PGON, 2>(a, nchunk, s);
}

template <typename T, typename C, int MODE, bool PGON> int occupancy_mode() {
  constexpr size_t smem = smem_bytes<C, PGON>();
  if (cudaFuncSetAttribute(k_pg<T, C, MODE, PGON, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 1;
  int blocks = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_pg<T, C, MODE, PGON, false, 2>, NT, smem) !=
      cudaSuccess)
    return 1;
  return blocks < 1 ? 1 : blocks;
}

}  // namespace

// The upwind scheme (pg = 0) reaches one node upstream and needs no staged
// tile: it runs in the streaming kernel of k_upres.cu.
template <typename T, typename C>
cudaError_t launch_pg(const PgArgs<T, C>& a, int mode, bool pg, int nchunk, cudaStream_t s) {
  if (pg && a.order == 3) return launch_pgd<T, C>(a, mode, nchunk, s);  // cubic: halo 9, direct passes
  if constexpr (std::is_same<T, float>::value && std::is_same<C, float>::value) {
    if (pg && pg2_applies(a)) return launch_pg2(a, mode, nchunk, s);  // FP32: direction pairs
  }
  if (pg)
    return mode == PG_RESID ? launch_mode<T, C, PG_RESID, true>(a, nchunk, s)
                            : launch_mode<T, C, PG_JACOBI, true>(a, nchunk, s);
  return launch_upres<T, C>(a, mode, nchunk, s);
}

template <typename T, typename C> int pg_blocks_per_sm(bool pg) {
  if constexpr (std::is_same<T, float>::value && std::is_same<C, float>::value) {
    if (pg) return pg2_blocks_per_sm();
  }
  return pg ? occupancy_mode<T, C, PG_JACOBI, true>() : upres_blocks_per_sm<T, C>();
}

template cudaError_t launch_pg<double, double>(const PgArgs<double, double>&, int, bool, int, cudaStream_t);
template cudaError_t launch_pg<float, float>(const PgArgs<float, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_pg<__nv_bfloat16, float>(const PgArgs<__nv_bfloat16, float>&, int, bool, int,
                                                     cudaStream_t);
template cudaError_t launch_pg<__half, float>(const PgArgs<__half, float>&, int, bool, int, cudaStream_t);
template int pg_blocks_per_sm<double, double>(bool);
template int pg_blocks_per_sm<float, float>(bool);
template int pg_blocks_per_sm<__nv_bfloat16, float>(bool);
template int pg_blocks_per_sm<__half, float>(bool);

}  // namespace btmg
