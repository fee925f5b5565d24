// btmg_common.cuh -- types and launcher declarations shared by the CUDA
// translation units of the btmg library (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>
#include <utility>

namespace btmg {

// ------------------------------------------- programmatic dependent launch -
// The kernels of a cycle are launched with programmatic stream
// serialisation: a kernel may be scheduled while its predecessor in the
// stream drains, so its launch overlaps the predecessor's last wave.
// pdl_wait() (first statement of such a kernel) blocks until the
// predecessor has completed and its writes are visible; pdl_launch() then
// lets the successor be scheduled.  Both are no-ops for a plain launch.
// BTMG_PDL=0 in the environment launches plainly.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("BTMG_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}
template <typename... KP, typename... A>
inline cudaError_t launch_pdl(void (*kern)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// ---------------------------------------------------------------- types ---
template <typename T> struct Conv;
template <> struct Conv<double> {
  __device__ __forceinline__ static double ld(const double* p) { return *p; }
  template <typename C> __device__ __forceinline__ static void st(double* p, C v) { *p = (double)v; }
};
template <> struct Conv<float> {
  __device__ __forceinline__ static float ld(const float* p) { return *p; }
  template <typename C> __device__ __forceinline__ static void st(float* p, C v) { *p = (float)v; }
};
template <> struct Conv<__nv_bfloat16> {
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  template <typename C> __device__ __forceinline__ static void st(__nv_bfloat16* p, C v) {
    *p = __float2bfloat16_rn((float)v);
  }
};
template <> struct Conv<__half> {
  __device__ __forceinline__ static float ld(const __half* p) { return __half2float(*p); }
  template <typename C> __device__ __forceinline__ static void st(__half* p, C v) {
    *p = __float2half_rn((float)v);
  }
};
// value of v after a round trip through storage type T (the stored value)
template <typename T, typename C> __device__ __forceinline__ C stored(C v) {
  T t;
  Conv<T>::st(&t, v);
  return (C)Conv<T>::ld(&t);
}

// Per-direction constants of one level (mu, nu, p and the upwind factors
// |mu|/dX, |nu|/dY), in the compute type.
template <typename C> struct Dir {
  C mu, nu, w, ax, ay;
};

enum { BC_VACUUM = 0, BC_REFLECTIVE = 1 };

// Halo rule of Sec. 2.3: an out-of-domain position takes 0 when it lies on
// an incoming side of a vacuum boundary (mu > 0 at x < 0, mu < 0 at x >= nx,
// likewise in y), otherwise the value of the nearest interior node.
struct Bc {
  int xlo, xhi, ylo, yhi;
};
__device__ __forceinline__ bool halo_is_zero(const Bc& bc, int gx, int gy, int nx, int ny, bool sxp,
                                             bool syp) {
  return (gx < 0 && bc.xlo == BC_VACUUM && sxp) || (gx >= nx && bc.xhi == BC_VACUUM && !sxp) ||
         (gy < 0 && bc.ylo == BC_VACUUM && syp) || (gy >= ny && bc.yhi == BC_VACUUM && !syp);
}
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------------- PG residual -------
enum { PG_RESID = 0, PG_JACOBI = 1 };

template <typename T, typename C> struct PgArgs {
  const T* psi;       // one group: [nd][ny][nx]
  T* psi_out;         // PG_JACOBI: updated angular flux, [nd][ny][nx]
  C* r_out;           // PG_RESID: residual b - A psi, [nd][ny][nx]
  const C* b;         // [ny][nx] isotropic right-hand side of this group
  const C* extra;     // nullable [nd][ny][nx] anisotropic source added to b
  const C* sigt;      // [ny][nx]
  const Dir<C>* dir;  // [nd]
  C* phi_part;        // PG_JACOBI: [nchunk][ny][nx] partial scalar fluxes
  C* rho_part;        // PG_RESID, nullable: [nchunk][ny][nx] partial sums of p_n r_n
  double* norm_part;  // PG_RESID: [gridDim.x*gridDim.y] partial sum p dx dy r^2
  int nx, ny, nd, dpc, tiles_x;  // dpc = directions per chunk
  C inv_dx, inv_dy, inv_dx2, inv_dy2, dx, dy, dxdy;
  C eps_k, a_kabs, a_ksq, a_r, half, beta;
  Bc bc;
  int* err;  // set to nonzero when a bounded wait gave up (device word)
  int order;  // ConvFEM order: 2 (quadratic) or 1 (linear) in the staged kernel, 3 (cubic) in k_pgd
  // cubic path (k_pgd.cu): 1D stencils m1, d1, s1 at offsets -3..3 and the
  // [nd][ny][nx] scratch of Psi_x, Psi_y, k_x, k_y
  C cm1[7], cd1[7], cs1[7];
  C *gpx, *gpy, *gkx, *gky;
  int chunk0;  // k_pg2: direction chunk of blockIdx.y = 0 (a launch over chunks chunk0 ..)
};

// ------------------------------------------------------- upwind Jacobi ----
enum { UP_CORR = 0, UP_UPDATE = 1 };
enum { INIT_ZERO = 0, INIT_UPSAMPLE = 1, INIT_SAME = 2 };

template <typename T, typename C> struct UpArgs {
  const C* src;        // [nd][ny][nx] source of the correction equation
  size_t src_stride;   // elements between direction planes of src (0: isotropic)
  const C* init;       // INIT_UPSAMPLE: coarse level [ndc][nyc][nxc]; INIT_SAME: [nd][ny][nx]
  C* delta_out;        // UP_CORR: [nd][ny][nx]
  const T* psi_in;     // UP_UPDATE
  T* psi_out;          // UP_UPDATE
  C* phi_part;         // UP_UPDATE: [nchunk][ny][nx]
  const C* sig;        // [ny][nx] (harmonic averaged on coarse levels)
  const Dir<C>* dir;   // [nd]
  const int* parent;   // INIT_UPSAMPLE: coarse direction of each direction [nd]
  int nx, ny, nr, nc, nd;
  int nxc, nyc, nrc, ncc;  // coarse dims (INIT_UPSAMPLE)
  int fx, fy, fr, fc;      // coarsening factors to the coarse level (1 or 2)
  int nu, init_mode, dpc, tiles_x;
  Bc bc;
  int* err;  // set to nonzero when a bounded wait gave up (device word)
};

// ----------------------------------------------------------- launchers -----
// All return cudaError_t of the launch.
template <typename T, typename C>
cudaError_t launch_upres(const PgArgs<T, C>& a, int mode, int nchunk, cudaStream_t s);
template <typename T, typename C> int upres_blocks_per_sm();
int upres_norm_blocks(int nx, int ny, int nchunk);  // norm partials of the upwind-mode kernel
cudaError_t launch_wait_selftest(int* err, int polls, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_pg(const PgArgs<T, C>& a, int mode, bool pg, int nchunk, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_pgd(const PgArgs<T, C>& a, int mode, int nchunk, cudaStream_t s);
// resident CTAs per SM of the PG kernel (for choosing whole-wave grids)
template <typename T, typename C> int pg_blocks_per_sm(bool pg);
// FP32 quadratic PG operator on direction pairs (k_pg2.cu): whether it takes
// these arguments (FP32 rows of a multiple of 4 nodes, even directions per
// chunk), its occupancy and its launch
bool pg2_applies(const PgArgs<float, float>& a);
int pg2_blocks_per_sm();
cudaError_t launch_pg2(const PgArgs<float, float>& a, int mode, int nchunk, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_upwind(const UpArgs<T, C>& a, int mode, int nchunk, cudaStream_t s);

// Scattering smoother (node-block Jacobi with in-node isotropic scattering;
// a variant of the upwind correction sweeps, k_scat.cu).
template <typename C> struct ScatArgs {
  const C* src;        // [nd][ny][nx] correction source
  size_t src_stride;   // elements between direction planes of src
  int init_mode;       // INIT_ZERO, INIT_UPSAMPLE (coarse, parent) or INIT_SAME (jin, cin)
  const C* jin;        // INIT_SAME: [nd][ny][nx] plain update J of the previous sweep
  const C* cin;        // INIT_SAME: [ny][nx] isotropic correction c of that sweep, or NULL
  const C* coarse;     // INIT_UPSAMPLE: coarser correction [ndc][nyc][nxc]
  const int* parent;   // INIT_UPSAMPLE: coarse direction of each direction [nd]
  int nxc, nyc, fx, fy;
  C* jout;             // [nd][ny][nx]
  C* part;             // [nchunk][ny][nx] sum of p_n J_n over each chunk
  const C* sig;        // [ny][nx]
  const Dir<C>* dir;   // [nd]
  int nx, ny, nd, dpc;
  Bc bc;
};
template <typename T, typename C> struct ScatFinal {
  const C* j;          // [nd][ny][nx] J of the last sweep (may alias delta_out)
  const C* c;          // [ny][nx] isotropic correction of the last sweep
  const C* sig;
  const Dir<C>* dir;
  int nx, ny, nd, dpc; // output chunking (dpc directions per block row)
  C* delta_out;        // delta = J + c / d, or NULL with psi_out set
  const T* psi_in;     // finest level: psi_out = psi_in + delta,
  T* psi_out;          //   scalar-flux partials of psi_out in phi_part
  C* phi_part;         //   [nchunk][ny][nx]
};
template <typename C> cudaError_t launch_scat_sweep(const ScatArgs<C>& a, int nchunk, cudaStream_t s);
template <typename C>
cudaError_t launch_scat_corr(const C* part, int nchunk, const C* w, int npix, C* c, cudaStream_t s);
template <typename T, typename C> cudaError_t launch_scat_final(const ScatFinal<T, C>& f, int nchunk, cudaStream_t s);
template <typename C>
cudaError_t launch_scat_gain(const C* sig, const C* crat, const Dir<C>* dir, int nd, int npix, C* w, cudaStream_t s);
// direction chunks of the sweeps on a level (csize: bytes of the compute
// type); scat_vec: whether its sweeps from J take four nodes per thread
int scat_chunks(int nx, int ny, int nd, int csize);
bool scat_vec(int nx, int csize);
// The coarsest levels, each of at most scat_tail_max<C>() unknowns, run in
// one single-CTA launch (k_tail): the restrictions down these levels, then
// their nu sweeps from the coarsest up, for the published cycle's upwind
// Jacobi (scat = 0) or the scattering smoother (scat = 1); lev[0] is the
// finest of them, its restricted residual an input.
constexpr int kScatTailLevels = 16;
template <typename C> constexpr int scat_tail_max() { return sizeof(C) == 8 ? 4096 : 8192; }
template <typename C> struct ScatTailLevel {
  C* s;               // [nd][ny][nx] restricted residual (written here for lev[1..])
  const C* rcoef;     // [nd] restriction weights to the next coarser level
  const C* w;         // [ny][nx] smoother gain (scat = 1)
  const C* sig;       // [ny][nx]
  const Dir<C>* dir;  // [nd]
  const int* parent;  // coarser-level direction of each direction (not for the coarsest)
  int nx, ny, nr, nc, nd, fx, fy, fr, fc;  // factors to the coarser level
};
template <typename C> struct ScatTail {
  ScatTailLevel<C> lev[kScatTailLevels];
  int count, nu, scat;
  Bc bc;
  C* out;  // delta of lev[0], [nd][ny][nx]
};
template <typename C> cudaError_t launch_scat_tail(const ScatTail<C>& t, cudaStream_t s);

// Batched coarse correction in one persistent launch (k_mg_impl.cuh): the
// restrictions and the upwind Jacobi sweeps of every level below the finest
// of every problem of a batch, as a queue of (segment, block) tasks.  A
// segment is one level's restriction or sweep of one problem; a task waits
// (bounded) until the previous segment of its problem is complete.  FP32.
struct CoarseRestrict {
  const float* fine;
  float* coarse;
  const float* rcoef;
  int nx, ny, nr, nc, nxc, nyc, nrc, ncc, fx, fy, fr, fc;
};
struct CoarseSeg {
  int type;    // 0 restriction, 1 upwind sweeps (UP_CORR)
  int arg;     // index into the restriction or sweep arguments
  int blocks;  // tasks of the segment
  int prev;    // segment of the same problem that must be complete first (-1: none)
  int tiles;   // sweeps: tiles of the level (task = tile + tiles * direction)
};
struct CoarseBatch {
  const CoarseSeg* seg;
  const int2* task;  // (segment, block) in an order where every prerequisite comes first
  int ntasks;
  const CoarseRestrict* ra;
  const UpArgs<float, float>* ua;
  unsigned* head;  // next task to take (zero before each launch)
  unsigned* done;  // finished tasks per segment (zero before each launch)
  int* err;        // set to nonzero when a bounded wait gave up
};
constexpr int kCoarseCells = 2048;  // coarse cells per restriction task
// sweeps per level nu (1..4) and tile width tu (16 or 32); ctas: CTAs per SM
bool coarse_batch_supported(int nu, int tu);
cudaError_t launch_coarse_batch(const CoarseBatch& cb, int nu, int tu, int ctas, cudaStream_t s);
constexpr size_t kCoarseWaitTestBytes = 1024;
cudaError_t launch_coarse_wait_selftest(void* ws, int* err, cudaStream_t s);

// particle balance of one group of an upwind-scheme solution (k_balance.cu):
// per-block FP64 partials (production, removal) and (x leakage, y leakage)
template <typename C>
cudaError_t launch_balance_volume(const C* src_g, const C* sigs_g, const C* sigt_g, const C* phi_part, int G, int g,
                                  int nchunk, int npix, double* part, int nblocks, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_balance_leak(const T* psi, const Dir<C>* dir, int nx, int ny, int nd, Bc bc, double dx, double dy,
                                double* part, int nblocks, cudaStream_t s);

template <typename C>
cudaError_t launch_restrict(const C* fine, C* coarse, const C* rcoef, int nx, int ny, int nr, int nc,
                            int nxc, int nyc, int nrc, int ncc, int fx, int fy, int fr, int fc,
                            cudaStream_t s);
template <typename C>
cudaError_t launch_prolong(const C* coarse, C* fine, int nx, int ny, int nr, int nc, int nxc, int nyc,
                           int nrc, int ncc, int fx, int fy, int fr, int fc, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_phi_partial(const T* psi, C* phi_part, const Dir<C>* dir, int nx, int ny, int nd,
                               int dpc, int nchunk, cudaStream_t s);
// b = s_g + sum_h sigma_s[g<-h] phi_h / (4 pi); qn2_part[block] = sum (b_fixed)^2
template <typename C>
cudaError_t launch_source(const C* src_g, const C* sigs_g /*[G][ny][nx] from h*/, const C* phi_part,
                          int G, int g, int nchunk, int npix, C* b, C* qfix_out, double* qn2_part,
                          int nblocks, cudaStream_t s);
template <typename C>
cudaError_t launch_phi_sum(const C* phi_part, int nchunk, int npix, C* phi, cudaStream_t s);
// out[0] = sum(part[0..n)) (deterministic, one block)
cudaError_t launch_sum(const double* part, int n, double* out, cudaStream_t s);
// FP32 restriction level 0 -> 1 of the fine residual r = r' + b assembled
// on the fly (r' = -A psi from a residual launch with zero source), r written
// back, with one norm partial p_n dx dy r^2 per CTA (k_mg_impl.cuh)
bool restrict_rb_applies(int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc, int ncc, int fx, int fy,
                         int fr, int fc, int max_parts, int* nparts);
cudaError_t launch_restrict_rb(float* r, const float* b, float* coarse, const float* rcoef, const Dir<float>* dir,
                               double dxdy, double* part, int nx, int ny, int nr, int nc, int nxc, int nyc, int nrc,
                               int ncc, cudaStream_t s);
// two such sums in one launch (each in launch_sum's order, so the same bits)
cudaError_t launch_sum2(const double* part_a, int na, double* out_a, const double* part_b, int nb, double* out_b,
                        cudaStream_t s);
// iterative refinement helpers: extra = alpha * r64 (to the compute type);
// psi64 += delta / alpha (delta in the storage type)
// learned correction: features [H8][W8][3] = (rho / rms(rho), log optical
// thickness, scattering ratio) from the residual-moment partials; apply
// psi_n += omega * scale * delta / (4 pi) and the flux partial of chunk 0
constexpr int kLearnFeatures = 4;  // input channels of the learned correction
constexpr int kLearnBlocks = 32;   // blocks of the coarse-canvas feature kernels
template <typename C>
cudaError_t launch_learn_features(const C* rho_part, int nchunk, const C* phi_part, const C* phi_prev, const C* sigt,
                                  const C* sigs_gg, double dx, int nx, int ny, int f, int W8, int H8, double* d_sum,
                                  double* d_part, float* feat, float* scale_out, cudaStream_t s);
template <typename C>
cudaError_t launch_dphi_norm(const C* phi_part, int nchunk, const C* phi_prev, int npix, double* d_part, int nblk,
                             double* out, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_learn_build(T* c_out, C* b_out, const float* delta, const C* sigt, const C* sigs_gg,
                               const Dir<C>* dir, int nd, int nx, int ny, int f, int W8, double dx, double dy,
                               double inv_len, cudaStream_t s);
template <typename C>
cudaError_t launch_learn_dot(const C* r1, const C* rc, const Dir<C>* dir, int nx, int ny, int nd, double dxdy,
                             double* part, int nblk, double* out, cudaStream_t s);
template <typename T, typename C>
cudaError_t launch_learn_update(T* psi, const T* c, size_t n, C* phi, const C* phi_c, size_t nphi, const double* ldot,
                                const double* rn2, double* stat, cudaStream_t s);
template <typename C>
cudaError_t launch_scale_to(const double* r64, C* extra, double alpha, size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_refine_update(double* psi64, const T* delta, double inv_alpha, size_t n, cudaStream_t s);

}  // namespace btmg
