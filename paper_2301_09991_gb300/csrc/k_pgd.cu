// k_pgd.cu -- the fine PG residual and PG Jacobi sweep (Eq. Petrov with the
// anisotropic nonlinear dissipation of Sec. 2.6; Eq. matrix_full with
// beta = 3) for the cubic ConvFEM order (7 x 7 filters, Sec. 2.7 and the
// Appendix), evaluated directly in three passes over global memory:
//   grad:  Psi_x = m1_y d1_x psi / dx,  Psi_y = d1_y m1_x psi / dy
//   k:     R_x = a_r mu (m1_x m1_y - I) Psi_x,
//          k_x = min(dx|mu|, a_kabs|R_x|dx/(eps+|Psi_x|), a_ksq R_x^2 dx/(eps+|mu|Psi_x^2))
//   apply: D_x = [s1_x m1_y (k_x psi) + k_x s1_x m1_y psi - psi s1_x m1_y k_x] / dx^2,
//          r = b - (mu Psi_x + nu Psi_y + half (D_x + D_y) + sigma_t psi)
// with the 1D stencils m1, d1, s1 of the order passed in the arguments
// (offsets -L..L).  Halo rule of Sec. 2.3 for psi (0 on an incoming vacuum
// side, otherwise the nearest interior node), nearest interior node for the
// derived fields.  Every filter here sums to zero except m1 (sum 1): the
// derivative taps act on psi - psi(node) and the (m1 m1 - I) taps on
// Psi - Psi(node), so FP32 rounds relative to the local variation; D is
// unchanged by a constant shift of psi, so its products use psi - psi(node)
// too.  The staged shared-memory kernel (k_pg.cu) covers orders 1 and 2;
// this path trades its speed for a halo of 9 nodes.
//
// Layout: 32 x 32 node tiles of 128 threads, a thread owning an 8-row strip
// of one column; grad and k run one direction per block row, apply a chunk
// of directions per block (scalar-flux and norm partials as in k_pg).
#include "btmg_common.cuh"

namespace btmg {
namespace {

constexpr int DT = 32;

template <typename C> __device__ __forceinline__ C dabs(C v) { return v < C(0) ? -v : v; }
__device__ __forceinline__ float ddiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return a / b; }

// psi with the halo rule of Sec. 2.3 (vacuum incoming side -> 0)
template <typename T, typename C>
__device__ __forceinline__ C psi_ext(const T* p, int x, int y, int nx, int ny, const Bc& bc, bool sxp, bool syp) {
  if ((x < 0 || x >= nx || y < 0 || y >= ny) && halo_is_zero(bc, x, y, nx, ny, sxp, syp)) return C(0);
  return (C)Conv<T>::ld(p + (size_t)clampi(y, 0, ny - 1) * nx + clampi(x, 0, nx - 1));
}
// derived field: nearest interior node
template <typename C> __device__ __forceinline__ C der_ext(const C* f, int x, int y, int nx, int ny) {
  return f[(size_t)clampi(y, 0, ny - 1) * nx + clampi(x, 0, nx - 1)];
}

// A thread owns an 8-row strip of one column (SR rows, 128 threads per
// 32 x 32 tile): the row sums of a 7-tap x pass are computed once per row and
// slide through a 7-deep register window for the y pass, so an output reads
// (SR + 2L) / SR rows of 7 taps instead of its full 49-point stencil.  Every
// shift below is constant along the strip (the first node's value): the
// filters it enters sum to zero or act through (m1 m1 - I), so the results
// are those of the definition.
constexpr int SR = 8, SNT = 128;

template <typename T, typename C, int L> __global__ void __launch_bounds__(SNT) k_pgd_grad(const PgArgs<T, C> a) {
  const int n = blockIdx.y;
  const int x = (blockIdx.x % a.tiles_x) * DT + (threadIdx.x & 31);
  const int ys = (blockIdx.x / a.tiles_x) * DT + (threadIdx.x >> 5) * SR;
  if (x >= a.nx || ys >= a.ny) return;
  const Dir<C> dr = a.dir[n];
  const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
  const size_t npix = (size_t)a.nx * a.ny;
  const T* pn = a.psi + (size_t)n * npix;
  const C c0 = (C)Conv<T>::ld(pn + (size_t)ys * a.nx + x);
  C wd[2 * L + 1], wm[2 * L + 1];  // row sums d1_x q and m1_x q of rows y - L .. y + L
#pragma unroll 1
  for (int r = 0; r < SR + 2 * L; ++r) {
    const int yr = ys - L + r;
    C sd = C(0), sm = C(0);
#pragma unroll
    for (int u = -L; u <= L; ++u) {
      const C q = psi_ext<T, C>(pn, x + u, yr, a.nx, a.ny, a.bc, sxp, syp) - c0;
      sd += a.cd1[u + L] * q;
      sm += a.cm1[u + L] * q;
    }
#pragma unroll
    for (int k = 0; k < 2 * L; ++k) wd[k] = wd[k + 1], wm[k] = wm[k + 1];
    wd[2 * L] = sd;
    wm[2 * L] = sm;
    if (r >= 2 * L) {
      const int y = yr - L;
      if (y < a.ny) {
        C gx = C(0), gy = C(0);
#pragma unroll
        for (int v = 0; v <= 2 * L; ++v) {
          gx += a.cm1[v] * wd[v];
          gy += a.cd1[v] * wm[v];
        }
        const size_t gi = (size_t)n * npix + (size_t)y * a.nx + x;
        a.gpx[gi] = gx * a.inv_dx;
        a.gpy[gi] = gy * a.inv_dy;
      }
    }
  }
}

template <typename T, typename C, int L> __global__ void __launch_bounds__(SNT) k_pgd_k(const PgArgs<T, C> a) {
  const int n = blockIdx.y;
  const int x = (blockIdx.x % a.tiles_x) * DT + (threadIdx.x & 31);
  const int ys = (blockIdx.x / a.tiles_x) * DT + (threadIdx.x >> 5) * SR;
  if (x >= a.nx || ys >= a.ny) return;
  const Dir<C> dr = a.dir[n];
  const size_t npix = (size_t)a.nx * a.ny;
  const C* px = a.gpx + (size_t)n * npix;
  const C* py = a.gpy + (size_t)n * npix;
  const C amu = dabs(dr.mu), anu = dabs(dr.nu);
  const C cx = px[(size_t)ys * a.nx + x], cy = py[(size_t)ys * a.nx + x];
  C wx[2 * L + 1], wy[2 * L + 1];  // row sums m1_x (Psi - c) of rows y - L .. y + L
#pragma unroll 1
  for (int r = 0; r < SR + 2 * L; ++r) {
    const int yr = ys - L + r;
    C sx = C(0), sy = C(0);
#pragma unroll
    for (int u = -L; u <= L; ++u) {
      sx += a.cm1[u + L] * (der_ext(px, x + u, yr, a.nx, a.ny) - cx);
      sy += a.cm1[u + L] * (der_ext(py, x + u, yr, a.nx, a.ny) - cy);
    }
#pragma unroll
    for (int k = 0; k < 2 * L; ++k) wx[k] = wx[k + 1], wy[k] = wy[k + 1];
    wx[2 * L] = sx;
    wy[2 * L] = sy;
    if (r >= 2 * L) {
      const int y = yr - L;
      if (y < a.ny) {
        const size_t i = (size_t)y * a.nx + x;
        const C px0 = px[i], py0 = py[i];
        C mx = C(0), my = C(0);
#pragma unroll
        for (int v = 0; v <= 2 * L; ++v) {
          mx += a.cm1[v] * wx[v];
          my += a.cm1[v] * wy[v];
        }
        const C Rx = a.a_r * dr.mu * (mx - (px0 - cx)), Ry = a.a_r * dr.nu * (my - (py0 - cy));
        const C kxa = ddiv(a.a_kabs * dabs(Rx) * a.dx, a.eps_k + dabs(px0));
        const C kya = ddiv(a.a_kabs * dabs(Ry) * a.dy, a.eps_k + dabs(py0));
        const C kxs = ddiv(a.a_ksq * Rx * Rx * a.dx, a.eps_k + amu * px0 * px0);
        const C kys = ddiv(a.a_ksq * Ry * Ry * a.dy, a.eps_k + anu * py0 * py0);
        const C kxm = a.dx * amu, kym = a.dy * anu;
        const size_t gi = (size_t)n * npix + i;
        a.gkx[gi] = kxm < kxa ? (kxm < kxs ? kxm : kxs) : (kxa < kxs ? kxa : kxs);
        a.gky[gi] = kym < kya ? (kym < kys ? kym : kys) : (kya < kys ? kya : kys);
      }
    }
  }
}

template <typename T, typename C, int MODE, int L>
__global__ void __launch_bounds__(SNT) k_pgd_apply(const PgArgs<T, C> a) {
  __shared__ double red[SNT / 32];
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int x = (tile % a.tiles_x) * DT + (threadIdx.x & 31);
  const int ys = (tile / a.tiles_x) * DT + (threadIdx.x >> 5) * SR;
  const size_t npix = (size_t)a.nx * a.ny;
  const int n_begin = chunk * a.dpc, n_end = min(n_begin + a.dpc, a.nd);
  double nrm = 0.0;
  C acc[SR];
#pragma unroll
  for (int k = 0; k < SR; ++k) acc[k] = C(0);
  const bool live = x < a.nx && ys < a.ny;
  if (live) {
    for (int n = n_begin; n < n_end; ++n) {
      const Dir<C> dr = a.dir[n];
      const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
      const T* pn = a.psi + (size_t)n * npix;
      const C* kxn = a.gkx + (size_t)n * npix;
      const C* kyn = a.gky + (size_t)n * npix;
      const C c0 = (C)Conv<T>::ld(pn + (size_t)ys * a.nx + x);
      // row sums of rows y - L .. y + L: s1_x (k_x q), s1_x q, s1_x k_x and
      // m1_x (k_y q), m1_x q, m1_x k_y, with q = psi - c0
      C w1[2 * L + 1], w2[2 * L + 1], w3[2 * L + 1], w4[2 * L + 1], w5[2 * L + 1], w6[2 * L + 1];
      C nrm_dir = C(0);
#pragma unroll 1
      for (int r = 0; r < SR + 2 * L; ++r) {
        const int yr = ys - L + r;
        C s1a = C(0), s1b = C(0), s1c = C(0), m1a = C(0), m1b = C(0), m1c = C(0);
#pragma unroll
        for (int u = -L; u <= L; ++u) {
          const C q = psi_ext<T, C>(pn, x + u, yr, a.nx, a.ny, a.bc, sxp, syp) - c0;
          const C kxe = der_ext(kxn, x + u, yr, a.nx, a.ny), kye = der_ext(kyn, x + u, yr, a.nx, a.ny);
          s1a += a.cs1[u + L] * (kxe * q);
          s1b += a.cs1[u + L] * q;
          s1c += a.cs1[u + L] * kxe;
          m1a += a.cm1[u + L] * (kye * q);
          m1b += a.cm1[u + L] * q;
          m1c += a.cm1[u + L] * kye;
        }
#pragma unroll
        for (int k = 0; k < 2 * L; ++k)
          w1[k] = w1[k + 1], w2[k] = w2[k + 1], w3[k] = w3[k + 1], w4[k] = w4[k + 1], w5[k] = w5[k + 1],
          w6[k] = w6[k + 1];
        w1[2 * L] = s1a, w2[2 * L] = s1b, w3[2 * L] = s1c, w4[2 * L] = m1a, w5[2 * L] = m1b, w6[2 * L] = m1c;
        if (r >= 2 * L) {
          const int y = yr - L;
          if (y < a.ny) {
            const size_t i = (size_t)y * a.nx + x, gi = (size_t)n * npix + i;
            const C p0 = (C)Conv<T>::ld(pn + i), q0 = p0 - c0;
            const C kx0 = kxn[i], ky0 = kyn[i];
            C fkx = C(0), fpx = C(0), fxk = C(0), fky = C(0), fpy = C(0), fyk = C(0);
#pragma unroll
            for (int v = 0; v <= 2 * L; ++v) {
              fkx += a.cm1[v] * w1[v];
              fpx += a.cm1[v] * w2[v];
              fxk += a.cm1[v] * w3[v];
              fky += a.cs1[v] * w4[v];
              fpy += a.cs1[v] * w5[v];
              fyk += a.cs1[v] * w6[v];
            }
            const C Dx = (fkx + kx0 * fpx - q0 * fxk) * a.inv_dx2;
            const C Dy = (fky + ky0 * fpy - q0 * fyk) * a.inv_dy2;
            const C sig = a.sigt[i];
            const C Apsi = dr.mu * a.gpx[gi] + dr.nu * a.gpy[gi] + a.half * (Dx + Dy) + sig * p0;
            const C res = a.b[i] + (a.extra ? a.extra[gi] : C(0)) - Apsi;
            const int k = r - 2 * L;
            if (MODE == PG_RESID) {
              a.r_out[gi] = res;
              nrm_dir += res * res;
              acc[k] += dr.w * res;
            } else {
              const C pnew = p0 + ddiv(res, a.beta * (dr.ax + dr.ay + sig));
              Conv<T>::st(a.psi_out + gi, pnew);
              acc[k] += dr.w * stored<T, C>(pnew);
            }
          }
        }
      }
      if (MODE == PG_RESID) nrm += (double)dr.w * (double)nrm_dir;
    }
    C* part = MODE == PG_JACOBI ? a.phi_part : a.rho_part;
    if (part) {
#pragma unroll
      for (int k = 0; k < SR; ++k) {
        const int y = ys + k;
        if (y < a.ny) part[(size_t)chunk * npix + (size_t)y * a.nx + x] = acc[k];
      }
    }
  }
  if (MODE == PG_RESID) {
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < SNT / 32; ++w) s += red[w];
      a.norm_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s * (double)a.dxdy;
    }
  }
}

}  // namespace

// Needs a.gpx, a.gpy, a.gkx, a.gky: [nd][ny][nx] scratch of the compute type.
template <typename T, typename C>
cudaError_t launch_pgd(const PgArgs<T, C>& a, int mode, int nchunk, cudaStream_t s) {
  if (a.order != 3) return cudaErrorNotSupported;
  const int tiles_y = (a.ny + DT - 1) / DT;
  const dim3 gdir(a.tiles_x * tiles_y, a.nd), gchunk(a.tiles_x * tiles_y, nchunk);
  k_pgd_grad<T, C, 3><<<gdir, SNT, 0, s>>>(a);
  k_pgd_k<T, C, 3><<<gdir, SNT, 0, s>>>(a);
  if (mode == PG_RESID)
    k_pgd_apply<T, C, PG_RESID, 3><<<gchunk, SNT, 0, s>>>(a);
  else
    k_pgd_apply<T, C, PG_JACOBI, 3><<<gchunk, SNT, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_pgd<double, double>(const PgArgs<double, double>&, int, int, cudaStream_t);
template cudaError_t launch_pgd<float, float>(const PgArgs<float, float>&, int, int, cudaStream_t);
template cudaError_t launch_pgd<__nv_bfloat16, float>(const PgArgs<__nv_bfloat16, float>&, int, int, cudaStream_t);
template cudaError_t launch_pgd<__half, float>(const PgArgs<__half, float>&, int, int, cudaStream_t);

}  // namespace btmg
