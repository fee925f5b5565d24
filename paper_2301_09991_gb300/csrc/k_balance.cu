// k_balance.cu -- particle balance of one group of a solution of the upwind
// fine scheme (Sec. 2.3 with the upwind filters of Sec. 2.4; pg = 0): the
// streaming term of the scheme telescopes over each row and column, so the
// converged discrete equations balance exactly, per group g,
//   production = dxdy sum_x (4 pi s_g + sum_{h != g} sigma_s[g<-h] phi_h)
//   removal    = dxdy sum_x (sigma_t,g - sigma_s[g<-g]) phi_g
//   leakage    = sum_n p_n ( |mu_n| dy sum_y (psi_n(x_out) - psi_n,halo(x_in))
//                          + |nu_n| dx sum_x (psi_n(y_out) - psi_n,halo(y_in)) )
// (phi = sum_n p_n psi_n, R3), where x_out is the downstream boundary column
// of direction n and psi_halo the incoming halo value of Sec. 2.3: 0 on a
// vacuum side, the boundary node's own value on a reflective one.  FP64
// accumulation; per-block partial sums (deterministic, no atomics).
#include "btmg_common.cuh"

namespace btmg {
namespace {

constexpr int BT = 256;

__device__ __forceinline__ void block_sum2(double a, double b, double* out_a, double* out_b) {
  __shared__ double ra[BT / 32], rb[BT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) ra[threadIdx.x >> 5] = a, rb[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < BT / 32; ++w) sa += ra[w], sb += rb[w];
    *out_a = sa;
    *out_b = sb;
  }
}

// production and removal partials of group g (phi from the direction-chunk
// partials of every group)
template <typename C>
__global__ void __launch_bounds__(BT) k_balance_volume(const C* __restrict__ src_g, const C* __restrict__ sigs_g,
                                                       const C* __restrict__ sigt_g, const C* __restrict__ phi_part,
                                                       int G, int g, int nchunk, int npix, double* __restrict__ part) {
  double prod = 0.0, rem = 0.0;
  for (int pix = blockIdx.x * BT + threadIdx.x; pix < npix; pix += gridDim.x * BT) {
    double in = 4.0 * 3.14159265358979323846 * (double)src_g[pix];
    for (int h = 0; h < G; ++h) {
      double phi = 0.0;
      for (int c = 0; c < nchunk; ++c) phi += (double)phi_part[((size_t)h * nchunk + c) * npix + pix];
      const double sg = (double)sigs_g[(size_t)h * npix + pix];
      if (h == g)
        rem += ((double)sigt_g[pix] - sg) * phi;
      else
        in += sg * phi;
    }
    prod += in;
  }
  block_sum2(prod, rem, &part[2 * blockIdx.x], &part[2 * blockIdx.x + 1]);
}

// leakage partials of one group: item = (direction, boundary index); the x
// faces carry ny items per direction, the y faces nx
template <typename T, typename C>
__global__ void __launch_bounds__(BT) k_balance_leak(const T* __restrict__ psi, const Dir<C>* __restrict__ dir, int nx,
                                                     int ny, int nd, Bc bc, double dx, double dy,
                                                     double* __restrict__ part) {
  const size_t npix = (size_t)nx * ny;
  const long long per_dir = (long long)nx + ny, total = per_dir * nd;
  double lx = 0.0, ly = 0.0;
  for (long long it = blockIdx.x * (long long)BT + threadIdx.x; it < total; it += (long long)gridDim.x * BT) {
    const int n = (int)(it / per_dir), k = (int)(it % per_dir);
    const Dir<C> d = dir[n];
    const T* pn = psi + (size_t)n * npix;
    if (k < ny) {  // x faces of row k
      const bool sxp = d.mu > C(0);
      const int xo = sxp ? nx - 1 : 0, xi = sxp ? 0 : nx - 1;  // outgoing and incoming boundary columns
      const bool vac_in = (sxp ? bc.xlo : bc.xhi) == BC_VACUUM;
      const double out = (double)Conv<T>::ld(pn + (size_t)k * nx + xo);
      const double in = vac_in ? 0.0 : (double)Conv<T>::ld(pn + (size_t)k * nx + xi);
      lx += (double)d.w * fabs((double)d.mu) * dy * (out - in);
    } else {  // y faces of column k - ny
      const int x = k - ny;
      const bool syp = d.nu > C(0);
      const int yo = syp ? ny - 1 : 0, yi = syp ? 0 : ny - 1;
      const bool vac_in = (syp ? bc.ylo : bc.yhi) == BC_VACUUM;
      const double out = (double)Conv<T>::ld(pn + (size_t)yo * nx + x);
      const double in = vac_in ? 0.0 : (double)Conv<T>::ld(pn + (size_t)yi * nx + x);
      ly += (double)d.w * fabs((double)d.nu) * dx * (out - in);
    }
  }
  block_sum2(lx, ly, &part[2 * blockIdx.x], &part[2 * blockIdx.x + 1]);
}

}  // namespace

template <typename C>
cudaError_t launch_balance_volume(const C* src_g, const C* sigs_g, const C* sigt_g, const C* phi_part, int G, int g,
                                  int nchunk, int npix, double* part, int nblocks, cudaStream_t s) {
  k_balance_volume<C><<<nblocks, BT, 0, s>>>(src_g, sigs_g, sigt_g, phi_part, G, g, nchunk, npix, part);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t launch_balance_leak(const T* psi, const Dir<C>* dir, int nx, int ny, int nd, Bc bc, double dx, double dy,
                                double* part, int nblocks, cudaStream_t s) {
  k_balance_leak<T, C><<<nblocks, BT, 0, s>>>(psi, dir, nx, ny, nd, bc, dx, dy, part);
  return cudaGetLastError();
}

template cudaError_t launch_balance_volume<double>(const double*, const double*, const double*, const double*, int,
                                                   int, int, int, double*, int, cudaStream_t);
template cudaError_t launch_balance_volume<float>(const float*, const float*, const float*, const float*, int, int,
                                                  int, int, double*, int, cudaStream_t);
template cudaError_t launch_balance_leak<double, double>(const double*, const Dir<double>*, int, int, int, Bc, double,
                                                         double, double*, int, cudaStream_t);
template cudaError_t launch_balance_leak<float, float>(const float*, const Dir<float>*, int, int, int, Bc, double,
                                                       double, double*, int, cudaStream_t);
template cudaError_t launch_balance_leak<__nv_bfloat16, float>(const __nv_bfloat16*, const Dir<float>*, int, int, int,
                                                               Bc, double, double, double*, int, cudaStream_t);
template cudaError_t launch_balance_leak<__half, float>(const __half*, const Dir<float>*, int, int, int, Bc, double,
                                                        double, double*, int, cudaStream_t);

}  // namespace btmg
