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
// Layout: 32 x 32 node tiles of 256 threads, a thread owning column tx and
// rows ty + 8k; grad and k run one direction per block row, apply a chunk
// of directions per block (scalar-flux and norm partials as in k_pg).
#include "btmg_common.cuh"

namespace btmg {
namespace {

constexpr int DT = 32, DNT = 256;

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

template <typename T, typename C, int L> __global__ void __launch_bounds__(DNT) k_pgd_grad(const PgArgs<T, C> a) {
  const int n = blockIdx.y;
  const int x = (blockIdx.x % a.tiles_x) * DT + (threadIdx.x & 31);
  const int y0 = (blockIdx.x / a.tiles_x) * DT + (threadIdx.x >> 5);
  if (x >= a.nx) return;
  const Dir<C> dr = a.dir[n];
  const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
  const size_t npix = (size_t)a.nx * a.ny;
  const T* pn = a.psi + (size_t)n * npix;
  for (int y = y0; y < min(y0 + DT, a.ny); y += 8) {
    const C c0 = (C)Conv<T>::ld(pn + (size_t)y * a.nx + x);
    C gx = C(0), gy = C(0);
#pragma unroll
    for (int v = -L; v <= L; ++v) {
      C sd = C(0), sm = C(0);  // d1_x and m1_x of row y + v
#pragma unroll
      for (int u = -L; u <= L; ++u) {
        const C q = psi_ext<T, C>(pn, x + u, y + v, a.nx, a.ny, a.bc, sxp, syp) - c0;
        sd += a.cd1[u + L] * q;
        sm += a.cm1[u + L] * q;
      }
      gx += a.cm1[v + L] * sd;
      gy += a.cd1[v + L] * sm;
    }
    const size_t gi = (size_t)n * npix + (size_t)y * a.nx + x;
    a.gpx[gi] = gx * a.inv_dx;
    a.gpy[gi] = gy * a.inv_dy;
  }
}

template <typename T, typename C, int L> __global__ void __launch_bounds__(DNT) k_pgd_k(const PgArgs<T, C> a) {
  const int n = blockIdx.y;
  const int x = (blockIdx.x % a.tiles_x) * DT + (threadIdx.x & 31);
  const int y0 = (blockIdx.x / a.tiles_x) * DT + (threadIdx.x >> 5);
  if (x >= a.nx) return;
  const Dir<C> dr = a.dir[n];
  const size_t npix = (size_t)a.nx * a.ny;
  const C* px = a.gpx + (size_t)n * npix;
  const C* py = a.gpy + (size_t)n * npix;
  const C amu = dabs(dr.mu), anu = dabs(dr.nu);
  for (int y = y0; y < min(y0 + DT, a.ny); y += 8) {
    const size_t i = (size_t)y * a.nx + x;
    const C px0 = px[i], py0 = py[i];
    C mx = C(0), my = C(0);
#pragma unroll
    for (int v = -L; v <= L; ++v) {
      C rx = C(0), ry = C(0);
#pragma unroll
      for (int u = -L; u <= L; ++u) {
        rx += a.cm1[u + L] * (der_ext(px, x + u, y + v, a.nx, a.ny) - px0);
        ry += a.cm1[u + L] * (der_ext(py, x + u, y + v, a.nx, a.ny) - py0);
      }
      mx += a.cm1[v + L] * rx;
      my += a.cm1[v + L] * ry;
    }
    const C Rx = a.a_r * dr.mu * mx, Ry = a.a_r * dr.nu * my;
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

template <typename T, typename C, int MODE, int L>
__global__ void __launch_bounds__(DNT) k_pgd_apply(const PgArgs<T, C> a) {
  __shared__ double red[DNT / 32];
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int x = (tile % a.tiles_x) * DT + (threadIdx.x & 31);
  const int y0 = (tile / a.tiles_x) * DT + (threadIdx.x >> 5);
  const size_t npix = (size_t)a.nx * a.ny;
  const int n_begin = chunk * a.dpc, n_end = min(n_begin + a.dpc, a.nd);
  double nrm = 0.0;
  C acc[4] = {C(0), C(0), C(0), C(0)};
  if (x < a.nx) {
    for (int n = n_begin; n < n_end; ++n) {
      const Dir<C> dr = a.dir[n];
      const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
      const T* pn = a.psi + (size_t)n * npix;
      const C* kxn = a.gkx + (size_t)n * npix;
      const C* kyn = a.gky + (size_t)n * npix;
      C nrm_dir = C(0);
#pragma unroll 1
      for (int k = 0; k < 4; ++k) {
        const int y = y0 + 8 * k;
        if (y >= a.ny) break;
        const size_t i = (size_t)y * a.nx + x, gi = (size_t)n * npix + i;
        const C p0 = (C)Conv<T>::ld(pn + i);
        const C kx0 = kxn[i], ky0 = kyn[i];
        C fkx = C(0), fpx = C(0), fky = C(0), fpy = C(0);  // f(k q; w), f(q; w) with q = psi - p0
#pragma unroll
        for (int v = -L; v <= L; ++v) {
          C ax1 = C(0), ax2 = C(0), ay1 = C(0), ay2 = C(0);
#pragma unroll
          for (int u = -L; u <= L; ++u) {
            const C q = psi_ext<T, C>(pn, x + u, y + v, a.nx, a.ny, a.bc, sxp, syp) - p0;
            const C kxe = der_ext(kxn, x + u, y + v, a.nx, a.ny), kye = der_ext(kyn, x + u, y + v, a.nx, a.ny);
            ax1 += a.cs1[u + L] * (kxe * q);
            ax2 += a.cs1[u + L] * q;
            ay1 += a.cm1[u + L] * (kye * q);
            ay2 += a.cm1[u + L] * q;
          }
          fkx += a.cm1[v + L] * ax1;
          fpx += a.cm1[v + L] * ax2;
          fky += a.cs1[v + L] * ay1;
          fpy += a.cs1[v + L] * ay2;
        }
        const C Dx = (fkx + kx0 * fpx) * a.inv_dx2, Dy = (fky + ky0 * fpy) * a.inv_dy2;
        const C sig = a.sigt[i];
        const C Apsi = dr.mu * a.gpx[gi] + dr.nu * a.gpy[gi] + a.half * (Dx + Dy) + sig * p0;
        const C r = a.b[i] + (a.extra ? a.extra[gi] : C(0)) - Apsi;
        if (MODE == PG_RESID) {
          a.r_out[gi] = r;
          nrm_dir += r * r;
          acc[k] += dr.w * r;
        } else {
          const C pnew = p0 + ddiv(r, a.beta * (dr.ax + dr.ay + sig));
          Conv<T>::st(a.psi_out + gi, pnew);
          acc[k] += dr.w * stored<T, C>(pnew);
        }
      }
      if (MODE == PG_RESID) nrm += (double)dr.w * (double)nrm_dir;
    }
    C* part = MODE == PG_JACOBI ? a.phi_part : a.rho_part;
    if (part) {
      for (int k = 0; k < 4; ++k) {
        const int y = y0 + 8 * k;
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
      for (int w = 0; w < DNT / 32; ++w) s += red[w];
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
  k_pgd_grad<T, C, 3><<<gdir, DNT, 0, s>>>(a);
  k_pgd_k<T, C, 3><<<gdir, DNT, 0, s>>>(a);
  if (mode == PG_RESID)
    k_pgd_apply<T, C, PG_RESID, 3><<<gchunk, DNT, 0, s>>>(a);
  else
    k_pgd_apply<T, C, PG_JACOBI, 3><<<gchunk, DNT, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_pgd<double, double>(const PgArgs<double, double>&, int, int, cudaStream_t);
template cudaError_t launch_pgd<float, float>(const PgArgs<float, float>&, int, int, cudaStream_t);
template cudaError_t launch_pgd<__nv_bfloat16, float>(const PgArgs<__nv_bfloat16, float>&, int, int, cudaStream_t);
template cudaError_t launch_pgd<__half, float>(const PgArgs<__half, float>&, int, int, cudaStream_t);

}  // namespace btmg
