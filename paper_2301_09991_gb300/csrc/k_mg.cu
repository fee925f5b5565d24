// k_mg.cu -- the HBM-bound multigrid kernels:
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
#include "btmg_common.cuh"

namespace btmg {
namespace {

constexpr int UT = 32, UNT = 256, NUMAX = 8;

template <typename T, typename C, int MODE>
__global__ void __launch_bounds__(UNT) k_upwind(const UpArgs<T, C> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nu = a.nu;
  const int W = UT + nu;          // loaded region (tile + nu upwind nodes)
  const int WS = UT + 2 * nu;     // sigma region covering both upwind sides
  C* D0 = reinterpret_cast<C*>(smem_raw);
  C* D1 = D0 + W * W;
  C* S = D1 + W * W;
  C* SG = S + W * W;

  const int tid = threadIdx.x;
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int x0 = (tile % a.tiles_x) * UT, y0 = (tile / a.tiles_x) * UT;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;

  for (int i = tid; i < WS * WS; i += UNT) {
    const int gx = x0 - nu + i % WS, gy = y0 - nu + i / WS;
    SG[i] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? a.sig[(size_t)gy * nx + gx] : C(0);
  }

  C phi_acc[(UT * UT) / UNT];
#pragma unroll
  for (int k = 0; k < (UT * UT) / UNT; ++k) phi_acc[k] = C(0);

  const int n_begin = chunk * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    const int ox = x0 - (sxp ? nu : 0), oy = y0 - (syp ? nu : 0);
    const int sgx = ox - (x0 - nu), sgy = oy - (y0 - nu);  // offset into SG
    const C* srcn = a.src + (size_t)n * a.src_stride;
    // parent direction and coarse plane for UpSamp
    int Np = 0;
    if (a.init_mode == INIT_UPSAMPLE) {
      const int per = a.nr * a.nc, f = n / per, j = (n % per) / a.nc, i = n % a.nc;
      Np = f * a.nrc * a.ncc + (j / a.fr) * a.ncc + i / a.fc;
    }
    __syncthreads();  // previous direction finished with D0/D1/S
    for (int i = tid; i < W * W; i += UNT) {
      const int lx = i % W, ly = i / W;
      const int gx = ox + lx, gy = oy + ly;
      C s = C(0), d = C(0);
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const size_t gi = (size_t)gy * nx + gx;
        s = srcn[gi];
        if (a.init_mode == INIT_UPSAMPLE)
          d = a.init[((size_t)Np * a.nyc + gy / a.fy) * a.nxc + gx / a.fx];
        else if (a.init_mode == INIT_SAME)
          d = a.init[(size_t)n * npix + gi];
      }
      S[i] = s;
      D0[i] = d;
    }
    __syncthreads();
    C* Dold = D0;
    C* Dnew = D1;
    const C ax = dr.ax, ay = dr.ay;
    const bool zx = sxp ? (a.bc.xlo == BC_VACUUM) : (a.bc.xhi == BC_VACUUM);
    const bool zy = syp ? (a.bc.ylo == BC_VACUUM) : (a.bc.yhi == BC_VACUUM);
    for (int k = 1; k <= nu; ++k) {
      const int xlo = sxp ? k : 0, xhi = sxp ? W : W - k;
      const int ylo = syp ? k : 0, yhi = syp ? W : W - k;
      for (int i = tid; i < W * W; i += UNT) {
        const int lx = i % W, ly = i / W;
        if (lx < xlo || lx >= xhi || ly < ylo || ly >= yhi) continue;
        const int gx = ox + lx, gy = oy + ly;
        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
        const C self = Dold[i];
        const bool bx = sxp ? (gx == 0) : (gx == nx - 1);  // upwind neighbour outside
        const bool by = syp ? (gy == 0) : (gy == ny - 1);
        const C ux = bx ? (zx ? C(0) : self) : Dold[i + (sxp ? -1 : 1)];
        const C uy = by ? (zy ? C(0) : self) : Dold[i + (syp ? -W : W)];
        const C sg = SG[(ly + sgy) * WS + lx + sgx];
        Dnew[i] = (S[i] + ax * ux + ay * uy) / (ax + ay + sg);
      }
      __syncthreads();
      C* t = Dold;
      Dold = Dnew;
      Dnew = t;
    }
    // store the tile
    const int tx0 = sxp ? nu : 0, ty0 = syp ? nu : 0;
#pragma unroll
    for (int k = 0; k < (UT * UT) / UNT; ++k) {
      const int i = tid + k * UNT;
      const int rx = i % UT, ry = i / UT;
      const int gx = x0 + rx, gy = y0 + ry;
      if (gx >= nx || gy >= ny) continue;
      const C d = Dold[(ry + ty0) * W + rx + tx0];
      const size_t gi = (size_t)n * npix + (size_t)gy * nx + gx;
      if (MODE == UP_CORR) {
        a.delta_out[gi] = d;
      } else {
        const C pn = Conv<T>::ld(a.psi_in + gi) + d;
        Conv<T>::st(a.psi_out + gi, pn);
        phi_acc[k] += dr.w * stored<T, C>(pn);
      }
    }
  }
  if (MODE == UP_UPDATE) {
    C* ph = a.phi_part + (size_t)chunk * npix;
#pragma unroll
    for (int k = 0; k < (UT * UT) / UNT; ++k) {
      const int i = tid + k * UNT;
      const int gx = x0 + i % UT, gy = y0 + i / UT;
      if (gx < nx && gy < ny) ph[(size_t)gy * nx + gx] = phi_acc[k];
    }
  }
}

template <typename C>
__global__ void k_restrict(const C* __restrict__ fine, C* __restrict__ coarse, const C* __restrict__ rcoef,
                           int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc, int ncc, int fx, int fy,
                           int fr, int fc) {
  const size_t total = (size_t)8 * nrc * ncc * nyc * nxc;
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total; id += (size_t)gridDim.x * blockDim.x) {
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
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < npix; pix += gridDim.x * blockDim.x) {
    C acc = C(0);
    for (int c = 0; c < nchunk; ++c) acc += part[(size_t)c * npix + pix];
    phi[pix] = acc;
  }
}

__global__ void k_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
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

inline int grid_for(size_t total, int threads) {
  size_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}

template <typename T, typename C, int MODE>
cudaError_t launch_up_mode(const UpArgs<T, C>& a, int nchunk, cudaStream_t s) {
  if (a.nu < 0 || a.nu > NUMAX) return cudaErrorInvalidValue;
  const int W = UT + a.nu, WS = UT + 2 * a.nu;
  const size_t smem = (3 * (size_t)W * W + (size_t)WS * WS) * sizeof(C);
  static bool attr_set = false;
  if (!attr_set) {
    const size_t maxs = (3 * (size_t)(UT + NUMAX) * (UT + NUMAX) + (size_t)(UT + 2 * NUMAX) * (UT + 2 * NUMAX)) * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_upwind<T, C, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxs);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tiles_y = (a.ny + UT - 1) / UT;
  dim3 grid(a.tiles_x * tiles_y, nchunk);
  k_upwind<T, C, MODE><<<grid, UNT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_upwind(const UpArgs<T, C>& a, int mode, int nchunk, cudaStream_t s) {
  return mode == UP_CORR ? launch_up_mode<T, C, UP_CORR>(a, nchunk, s) : launch_up_mode<T, C, UP_UPDATE>(a, nchunk, s);
}

template <typename C>
cudaError_t launch_restrict(const C* fine, C* coarse, const C* rcoef, int nx, int ny, int nr, int nc, int nxc,
                            int nyc, int nrc, int ncc, int fx, int fy, int fr, int fc, cudaStream_t s) {
  const size_t total = (size_t)8 * nrc * ncc * nyc * nxc;
  k_restrict<C><<<grid_for(total, 256), 256, 0, s>>>(fine, coarse, rcoef, nx, ny, nr, nc, nxc, nyc, nrc, ncc, fx,
                                                      fy, fr, fc);
  return cudaGetLastError();
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
  k_phi_partial<T, C><<<grid_for((size_t)nchunk * npix, 256), 256, 0, s>>>(psi, part, dir, npix, nd, dpc, nchunk);
  return cudaGetLastError();
}

template <typename C>
cudaError_t launch_source(const C* src_g, const C* sigs_g, const C* phi_part, int G, int g, int nchunk, int npix,
                          C* b, C* qfix, double* qn2_part, int nblocks, cudaStream_t s) {
  k_source<C><<<nblocks, 256, 0, s>>>(src_g, sigs_g, phi_part, G, g, nchunk, npix, b, qfix, qn2_part);
  return cudaGetLastError();
}

template <typename C>
cudaError_t launch_phi_sum(const C* part, int nchunk, int npix, C* phi, cudaStream_t s) {
  k_phi_sum<C><<<grid_for(npix, 256), 256, 0, s>>>(part, nchunk, npix, phi);
  return cudaGetLastError();
}

cudaError_t launch_sum(const double* part, int n, double* out, cudaStream_t s) {
  k_sum<<<1, 1024, 0, s>>>(part, n, out);
  return cudaGetLastError();
}

#define INST_TC(T, C)                                                                                     \
  template cudaError_t launch_upwind<T, C>(const UpArgs<T, C>&, int, int, cudaStream_t);                \
  template cudaError_t launch_phi_partial<T, C>(const T*, C*, const Dir<C>*, int, int, int, int, int, cudaStream_t);
INST_TC(double, double)
INST_TC(float, float)
INST_TC(__nv_bfloat16, float)
INST_TC(__half, float)
#define INST_C(C)                                                                                          \
  template cudaError_t launch_restrict<C>(const C*, C*, const C*, int, int, int, int, int, int, int, int, int, int, \
                                          int, int, cudaStream_t);                                         \
  template cudaError_t launch_prolong<C>(const C*, C*, int, int, int, int, int, int, int, int, int, int, int, int, \
                                         cudaStream_t);                                                    \
  template cudaError_t launch_source<C>(const C*, const C*, const C*, int, int, int, int, C*, C*, double*, int, \
                                        cudaStream_t);                                                     \
  template cudaError_t launch_phi_sum<C>(const C*, int, int, C*, cudaStream_t);
INST_C(double)
INST_C(float)

}  // namespace btmg
