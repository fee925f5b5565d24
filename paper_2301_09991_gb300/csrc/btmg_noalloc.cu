// btmg_noalloc.cu -- an allocation-free form of btmg_apply_operator.
//
// Some callers cannot allocate device memory: a host program or framework
// that reserves the GPU's memory up front for its own pool and gives every
// library a fixed budget (a cudaMalloc inside the library would fail or
// fragment that pool), a latency-critical loop in which cudaMalloc and
// cudaFree, which may synchronise the device, are not acceptable, or an
// embedded runtime that lends no device allocator to libraries.
// btmg_apply_operator_noalloc() serves them: the caller passes every input
// and output as device pointers, and the scratch the operator needs (scalar
// flux, assembled source, direction table, error word and the partial sums
// of the norms) lives in one file-scope device array of fixed size,
// g_scratch below.  Nothing here calls cudaMalloc, cudaFree or any
// allocating routine, and no host memory is copied to the device: the
// direction table is computed by a kernel.
//
// The array is part of the library image, so every GPU that loads the
// library holds it (BTMG_NOALLOC_SCRATCH_BYTES) until the process exits.
// All calls share it and it keeps the last call's contents; every byte a
// call reads is written by that same call first (the error word is cleared
// at the start of each call), but two calls that overlap on the GPU
// (different streams) race on it.
#include <cmath>
#include <cstdint>

#include "../../include/btmg.h"
#include "btmg_common.cuh"

using namespace btmg;

namespace {

constexpr int kMaxPix = BTMG_NOALLOC_MAX_NODES;
constexpr int kMaxDirs = BTMG_NOALLOC_MAX_DIRS;
constexpr int kTile = 32;
constexpr int kChunks = 16;  // direction chunks of the residual kernel
constexpr int kMaxNormParts = (kMaxPix / (kTile * kTile) + 64) * kChunks;
constexpr int kQBlocks = 1024;
// layout of the scratch array (offsets in bytes, each 256-byte aligned)
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffPhi = 0;
constexpr size_t kOffB = align256(kOffPhi + sizeof(float) * kMaxPix);
constexpr size_t kOffDir = align256(kOffB + sizeof(float) * kMaxPix);
constexpr size_t kOffNorm = align256(kOffDir + sizeof(Dir<float>) * kMaxDirs);
constexpr size_t kOffQ = align256(kOffNorm + sizeof(double) * kMaxNormParts);
constexpr size_t kOffSums = align256(kOffQ + sizeof(double) * kQBlocks);
constexpr size_t kOffErr = kOffSums + 2 * sizeof(double);
constexpr size_t kScratchBytes = align256(kOffErr + sizeof(int));
static_assert(kScratchBytes <= BTMG_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

__device__ __align__(256) unsigned char g_scratch[BTMG_NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch per device, looked up once per device (the
// host-side name g_scratch is only a stand-in for the device symbol).
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

// Octahedral directions (Sec. 2.2) of a level with nr x nc patches per
// face, in one block: thread i of face 0 integrates its patch's solid angle
// and first moments with 16 x 16 Gauss-Legendre points of the collapsed map
// X(u, t) = (1-t)((1-u) a + u b) + t c, whose solid-angle element is
// (1-t)/|X|^3; the other faces are the sign flips of face 0 (same areas,
// mirrored moments).  Weights are scaled so that they sum to 4 pi.
constexpr int kGauss = 16;
constexpr int kDirThreads = 256;  // >= nr * nc for every accepted size
__global__ void __launch_bounds__(kDirThreads) k_noalloc_directions(int nr, int nc, double dx, double dy,
                                                                   Dir<float>* out) {
  __shared__ double gx[kGauss], gw[kGauss], red[kDirThreads / 32];
  const int tid = threadIdx.x;
  if (tid < kGauss) {  // node tid of the 16-point rule: Newton on P_16 from a cosine guess
    const double pi = 3.14159265358979323846;
    double t = cos(pi * (4.0 * tid + 3.0) / (4.0 * kGauss + 2.0)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pm = 0.0, p = 1.0;
      for (int m = 1; m <= kGauss; ++m) {
        const double pn = ((2.0 * m - 1.0) * t * p - (m - 1.0) * pm) / m;
        pm = p;
        p = pn;
      }
      dp = kGauss * (pm - t * p) / (1.0 - t * t);
      const double step = p / dp;
      t -= step;
      if (fabs(step) < 1e-16) break;
    }
    gx[tid] = 0.5 * (1.0 + t);
    gw[tid] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
  __syncthreads();
  const int q = nr * nc;
  double area = 0.0, mx = 0.0, my = 0.0;
  if (tid < q) {
    const int j = tid / nc, i = tid % nc;
    for (int a = 0; a < kGauss; ++a)
      for (int b = 0; b < kGauss; ++b) {
        const double t = (j + gx[a]) / nr, u = (i + gx[b]) / nc;
        const double X0 = (1 - t) * (1 - u), X1 = (1 - t) * u, X2 = t;
        const double r2 = X0 * X0 + X1 * X1 + X2 * X2, r = sqrt(r2);
        const double dS = gw[a] * gw[b] / (double(nr) * nc) * (1 - t) / (r2 * r);
        area += dS;
        mx += dS * X0 / r;
        my += dS * X1 / r;
      }
  }
  double s = area;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  double face = 0.0;
  for (int w = 0; w < kDirThreads / 32; ++w) face += red[w];
  if (tid >= q) return;
  const double w = area * 4.0 * 3.14159265358979323846 / (8.0 * face);
  const double mu = mx / area, nu = my / area;
  for (int f = 0; f < 8; ++f) {
    const double sx = (f & 1) ? -1.0 : 1.0, sy = (f & 2) ? -1.0 : 1.0;
    Dir<float> d;
    d.mu = (float)(sx * mu);
    d.nu = (float)(sy * nu);
    d.w = (float)w;
    d.ax = (float)(mu / dx);
    d.ay = (float)(nu / dy);
    out[f * q + tid] = d;
  }
}

}  // namespace

extern "C" int btmg_apply_operator_noalloc(int32_t nx, int32_t ny, double lx, double ly, int32_t n_polar,
                                           int32_t n_azim, const int32_t bc[4], int32_t pg, int32_t pg_half,
                                           const float* sigma_t, const float* sigma_s, const float* source,
                                           const float* psi, float* r, void* stream, double* rel_resid) {
  if (nx < 1 || ny < 1 || !(lx > 0) || !(ly > 0) || !bc || !sigma_t || !sigma_s || !source || !psi || !r)
    return BTMG_ERR_INVALID_ARG;
  if (n_polar < 2 || n_polar % 2 || n_azim < 4 || n_azim % 4) return BTMG_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (bc[i] != BTMG_VACUUM && bc[i] != BTMG_REFLECTIVE) return BTMG_ERR_INVALID_ARG;
  const int nr = n_polar / 2, nc = n_azim / 4, nd = 8 * nr * nc;
  // sizes beyond the fixed scratch: a distinct status, nothing launched
  if ((int64_t)nx * ny > kMaxPix || nd > kMaxDirs) return BTMG_ERR_NOALLOC_TOO_LARGE;
  const int tiles_x = (nx + kTile - 1) / kTile;
  const int64_t tiles = (int64_t)tiles_x * ((ny + kTile - 1) / kTile);
  // norm partials written by the residual kernel: one per 32x32 tile and
  // chunk (PG), one per 128x8 tile and chunk (upwind scheme)
  auto parts = [&](int c) -> int64_t { return pg ? tiles * c : (int64_t)upres_norm_blocks(nx, ny, c); };
  int nchunk = kChunks;  // direction chunks of the residual kernel
  while (nchunk > 1 && (nd % nchunk || parts(nchunk) > kMaxNormParts)) nchunk >>= 1;
  if (parts(nchunk) > kMaxNormParts) return BTMG_ERR_NOALLOC_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BTMG_ERR_CUDA;
  if (!g_scratch_dev[dev]) {  // first call on this device: resolve the symbol
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return BTMG_ERR_CUDA;
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* base = g_scratch_dev[dev];
  float* phi = reinterpret_cast<float*>(base + kOffPhi);
  float* b = reinterpret_cast<float*>(base + kOffB);
  Dir<float>* dir = reinterpret_cast<Dir<float>*>(base + kOffDir);
  double* norm_part = reinterpret_cast<double*>(base + kOffNorm);
  double* q_part = reinterpret_cast<double*>(base + kOffQ);
  double* sums = reinterpret_cast<double*>(base + kOffSums);
  int* err = reinterpret_cast<int*>(base + kOffErr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const double dx = lx / nx, dy = ly / ny;
  if (nr * nc > kDirThreads) return BTMG_ERR_NOALLOC_TOO_LARGE;
  k_noalloc_directions<<<1, kDirThreads, 0, s>>>(nr, nc, dx, dy, dir);
  if (cudaGetLastError() != cudaSuccess) return BTMG_ERR_CUDA;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return BTMG_ERR_CUDA;
  // scalar flux in one chunk, then b = s + sigma_s phi / (4 pi)
  if (launch_phi_partial<float, float>(psi, phi, dir, nx, ny, nd, nd, 1, s) != cudaSuccess) return BTMG_ERR_CUDA;
  const int npix = nx * ny;
  const int qb = (npix + 255) / 256 < kQBlocks ? (npix + 255) / 256 : kQBlocks;
  if (launch_source<float>(source, sigma_s, phi, 1, 0, 1, npix, b, nullptr, rel_resid ? q_part : nullptr, qb, s) !=
      cudaSuccess)
    return BTMG_ERR_CUDA;
  PgArgs<float, float> a{};
  a.psi = psi;
  a.r_out = r;
  a.b = b;
  a.sigt = sigma_t;
  a.dir = dir;
  a.nx = nx;
  a.ny = ny;
  a.nd = nd;
  a.tiles_x = tiles_x;
  a.dpc = nd / nchunk;
  a.dx = (float)dx;
  a.dy = (float)dy;
  a.inv_dx = (float)(1.0 / dx);
  a.inv_dy = (float)(1.0 / dy);
  a.inv_dx2 = (float)(1.0 / (dx * dx));
  a.inv_dy2 = (float)(1.0 / (dy * dy));
  a.dxdy = (float)(dx * dy);
  a.eps_k = 1e-3f;
  a.a_kabs = 0.25f;
  a.a_ksq = 2.0f;
  a.order = 2;
  a.a_r = 3.0f;
  a.half = pg_half ? 0.5f : 1.0f;
  a.beta = 1.0f;
  a.bc = Bc{bc[0], bc[1], bc[2], bc[3]};
  a.norm_part = norm_part;
  a.err = err;
  if (launch_pg<float, float>(a, PG_RESID, pg != 0, nchunk, s) != cudaSuccess) return BTMG_ERR_CUDA;
  if (!rel_resid) return BTMG_OK;
  // ||r||_W / ||s||_W (W = p_n dx dy) from the kernels' partial sums, and
  // the error word, which a bounded wait that gave up has set
  if (launch_sum(norm_part, (int)parts(nchunk), sums, s) != cudaSuccess ||
      launch_sum(q_part, qb, sums + 1, s) != cudaSuccess)
    return BTMG_ERR_CUDA;
  double host[2];
  int host_err = 0;
  if (cudaMemcpyAsync(host, sums, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BTMG_ERR_CUDA;
  if (host_err) return BTMG_ERR_TIMEOUT;
  const double wq = 4.0 * 3.14159265358979323846 * dx * dy;
  *rel_resid = host[1] > 0 ? std::sqrt(host[0] / (wq * host[1])) : std::sqrt(host[0]);
  return BTMG_OK;
}
