/*
 * btmg.h -- C ABI of the GB300 (sm_103a) space-angle sawtooth multigrid
 * solver for the fixed-source 2D-space x 2D-angle discretised Boltzmann
 * transport equation (Phillips et al., arXiv 2301.09991).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status: BTMG_OK (0) or a negative BTMG_ERR_*.
 *    No C++ exception crosses the ABI.  btmg_error_string() names a status;
 *    btmg_last_error() gives a per-thread detail message for the last failure.
 *  - Angular-flux buffers (psi, r, corrections) and scalar-flux buffers are
 *    CALLER-OWNED DEVICE pointers (e.g. torch.Tensor.data_ptr()).  The library
 *    never frees or retains them beyond the call.  The library owns its
 *    workspaces and frees them in btmg_destroy_problem().
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are stream-ordered and asynchronous unless stated.
 *  - A problem handle is not thread-safe: one host thread at a time.
 *  - Layout of an angular flux with G groups on level l (level 0 = finest):
 *      psi[g][n][y][x], n = face*(nr*nc) + j*nc + i,
 *    dense, x fastest; face = 4*(xi<0) + 2*(nu<0) + (mu<0) is the octahedron
 *    face, j the polar and i the azimuthal patch index inside it (Sec. 2.2,
 *    Fig. octa).  btmg_get_layout() returns the strides.
 *  - Element type of psi is desc.psi_dtype.  Compute ("accumulation") type
 *    is FP64 for BTMG_F64 storage and FP32 otherwise; residuals, scalar
 *    fluxes and explicit sources passed to the library use the compute type.
 */
#ifndef BTMG_H
#define BTMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BTMG_OK 0
#define BTMG_ERR_INVALID_ARG (-1)
#define BTMG_ERR_CUDA (-2)
#define BTMG_ERR_OOM (-3)
#define BTMG_ERR_NOT_CONVERGED (-4)
#define BTMG_ERR_DIVERGED (-5)
#define BTMG_ERR_TIMEOUT (-6)
#define BTMG_ERR_NAN (-7)
#define BTMG_ERR_UNSUPPORTED (-8)

/* storage types of psi */
#define BTMG_F64 0
#define BTMG_F32 1
#define BTMG_BF16 2
#define BTMG_F16 3

/* boundary conditions (Sec. 2.1): vacuum psi = 0 on incoming directions;
 * reflective d psi / dn = 0 (halo copies the adjacent interior node). */
#define BTMG_VACUUM 0
#define BTMG_REFLECTIVE 1

/* smoother kinds for btmg_smooth */
#define BTMG_SMOOTH_UPWIND 0
#define BTMG_SMOOTH_PG 1

typedef struct btmg_problem btmg_problem;

/* Problem statement (Sec. 2.1, Eq. gov-simple; materials per region as in
 * Tab. sing_duct_data).  Nodes are cell centred, dx = lx/nx (Sec. 3.1).
 * All host arrays are copied by btmg_create_problem.                       */
typedef struct {
  int32_t nx, ny;          /* nodes in x and y (>= 1)                        */
  double lx, ly;           /* domain size (> 0)                              */
  int32_t order;           /* ConvFEM order: 2 (quadratic 5x5 filters), 1 (linear
                              3x3; PG in FP64/FP32 only) or 3 (cubic 7x7, halo 9:
                              direct-pass kernels with a 4 x psi-sized scratch) */
  int32_t n_polar, n_azim; /* direction grid: 8 faces of (n_polar/2)x(n_azim/4) */
  int32_t n_groups;        /* energy groups G (>= 1)                         */
  const int32_t* region;   /* host [ny][nx] region id per node               */
  int32_t n_regions;
  const double* sigma_t;   /* host [n_regions][G] total cross section        */
  const double* sigma_s;   /* host [n_regions][G][G] isotropic, [to g][from g'] */
  const double* source;    /* host [n_regions][G] isotropic source / steradian */
  int32_t bc[4];           /* xlo, xhi, ylo, yhi: BTMG_VACUUM / BTMG_REFLECTIVE */
  int32_t pg;              /* 1: nonlinear PG on the finest level; 0: upwind */
  int32_t nu_jacobi;       /* Jacobi sweeps per level (3), 1..8              */
  double beta_pg;          /* fine PG Jacobi diagonal factor (3.0)           */
  int32_t psi_dtype;       /* BTMG_F64 / BTMG_F32 / BTMG_BF16 / BTMG_F16     */
  int32_t max_levels;      /* 0: coarsen until every dimension is 1          */
  int32_t pg_half;         /* 1: scale f^{k-Diff} by 1/2 (analytic form)     */
  int32_t chunks;          /* direction chunks per group (CTAs along the
                              direction axis of the fine kernels): 0 picks the
                              count whose grid best fills whole waves of
                              resident CTAs; otherwise a divisor of the number
                              of directions, at most 64 (set by the batch
                              autotuner)                                     */
  int32_t scat_levels;     /* scattering smoother, a variant of the upwind
                              correction sweeps (the method as published has
                              none, Sec. 2.5): 0 off; 1 on the levels of the
                              coarsest angular resolution (N_r = N_c = 1);
                              2 on every level.  On those levels each node's
                              directions are solved together with the in-group
                              isotropic scattering sigma_s phi / (4 pi), upstream
                              neighbours lagged; coarse sigma_s = harmonic
                              sigma_t x the mean sigma_s / sigma_t of the
                              children.  Needs sigma_s,gg <= sigma_t.          */
} btmg_problem_desc;

typedef struct {
  int32_t cycles;        /* sawtooth cycles performed (all groups)           */
  int32_t status;        /* BTMG_OK, _NOT_CONVERGED, _DIVERGED or _NAN       */
  double rel_resid;      /* ||r||_W / ||q||_W of the returned psi (FP64)     */
  double* history;       /* optional caller host array, per-cycle residual   */
  int32_t history_len;   /* capacity of history (0 if NULL)                  */
  int32_t check_every;   /* read the residual back every this many cycles (0 -> 1) */
  int32_t max_outer;     /* passes over the groups (0: 1 without upscatter, else 8) */
} btmg_solve_info;

/* Builds the quadrature (Sec. 2.2), the space-angle hierarchy with harmonic
 * averaged cross sections (Sec. 2.5) and the device workspaces.  Copies every
 * host array.  Errors: INVALID_ARG (bad sizes, region ids, dtype, order outside 1..3, chunks,
 * a non-finite or negative cross section, a non-finite source, scat_levels
 * outside 0..2 or, with scat_levels, an in-group sigma_s above sigma_t),
 * UNSUPPORTED (pg = 1 with order 1 and BF16/FP16 storage), OOM, CUDA.
 * *out is NULL on failure.                                                 */
int btmg_create_problem(const btmg_problem_desc* desc, void* stream, btmg_problem** out);

/* Frees every library-owned device buffer.  NULL is accepted.              */
int btmg_destroy_problem(btmg_problem* p);

/* Total unknowns G * n_dirs * ny * nx of the finest level.                 */
int btmg_num_unknowns(const btmg_problem* p, int64_t* n);

/* Element strides of psi: [g, face, j, i, y, x].                           */
int btmg_get_layout(const btmg_problem* p, int64_t strides[6]);

/* Number of levels, and per level: dims = {nx, ny, nr, nc, n_dirs},
 * dxdy = {dX, dY} (Sec. 2.5).                                              */
int btmg_num_levels(const btmg_problem* p, int32_t* levels);
int btmg_level_info(const btmg_problem* p, int32_t level, int32_t dims[5], double dxdy[2]);

/* Directions of a level: mu, nu, p (host double arrays of n_dirs).         */
int btmg_level_quadrature(const btmg_problem* p, int32_t level, double* mu, double* nu,
                          double* w);

/* phi_g = sum_n p_n psi_{n,g} (Sec. 2.2).  psi: device [G][nd][ny][nx] of
 * psi_dtype; phi: device [G][ny][nx] of the compute type.                  */
int btmg_scalar_flux(btmg_problem* p, const void* psi, void* phi, void* stream);

/* r = b - A psi for every group (Eq. Petrov with the anisotropic nonlinear
 * PG dissipation of Sec. 2.6, or the upwind operator of Sec. 2.3 if pg = 0),
 * b = s + sum_g' sigma_s[g<-g'] phi_g' / (4 pi).  psi: device
 * [G][nd][ny][nx] psi_dtype; r: device, same shape, compute type.          */
int btmg_apply_operator(btmg_problem* p, const void* psi, void* r, void* stream);

/* Jacobi smoothing (Eq. matrix_full).
 *  kind = BTMG_SMOOTH_PG: level must be 0 and src NULL; `sweeps` fine PG
 *    Jacobi sweeps psi <- psi + (beta d)^{-1}(b - A psi) on the full problem
 *    (groups in order), psi device [G][nd][ny][nx].
 *  kind = BTMG_SMOOTH_UPWIND: `sweeps` Jacobi sweeps of the upwind system
 *    A_up,l psi = src of level `level` for group `group` (beta = 1, no
 *    scattering: the correction equation of the cycle; on the levels of the
 *    scattering smoother (desc.scat_levels) node-block sweeps of
 *    (A_up,l - sigma_s / (4 pi) sum_n p_n) psi = src instead); psi and src
 *    are device buffers of one group on that level, [nd_l][ny_l][nx_l], both
 *    of the compute type.                                                  */
int btmg_smooth(btmg_problem* p, void* psi, const void* src, int32_t level, int32_t group,
                int32_t sweeps, int32_t kind, void* stream);

/* Restriction level -> level+1 (Sec. 2.5): coarse = sum_children
 * p dx dy fine / (P dX dY).  Buffers of one group, compute type.           */
int btmg_restrict(btmg_problem* p, int32_t level, const void* fine, void* coarse, void* stream);

/* UpSamp level+1 -> level (Sec. 2.5): every fine unknown takes its coarse
 * parent's value.  Buffers of one group, compute type.                     */
int btmg_prolong(btmg_problem* p, int32_t level, const void* coarse, void* fine, void* stream);

/* One sawtooth cycle (Fig. multi_grid_it) per group, groups in order with
 * the latest scalar fluxes (block Gauss-Seidel).  psi updated in place.
 * rel_resid (nullable, host) receives ||r||_W/||q||_W of the INPUT psi
 * (FP64 reduction); if non-NULL the call synchronises the stream.          */
int btmg_mg_cycle(btmg_problem* p, void* psi, double* rel_resid, void* stream);

/* The same cycle (Fig. multi_grid_it) on psi in HOST memory: psi_in
 * ([G][nd][ny][nx], storage type, the btmg_get_layout order) is copied to a
 * device buffer that the problem owns (allocated by the first call, freed
 * with the problem), the cycle runs, and the result is written to psi_out
 * (host, same layout; may be psi_in).  With page-locked host buffers the
 * copies overlap kernels: each group's final PG Jacobi (FP32 paired kernel,
 * direction chunks a multiple of 4) runs as four launches over consecutive
 * direction ranges on side streams, every range copied back as soon as its
 * launch is done (other kernels copy a group while the next group cycles);
 * with one group on the paired kernel the copy in also arrives in four
 * ranges, each followed at once by its scalar-flux partials and its
 * residual with zero source, and the source is added in the restriction to
 * level 1.  rel_resid as in btmg_mg_cycle (then summed in another order:
 * equal to about 1e-8); with it the call returns when psi_out is complete,
 * without it psi_out is complete once `stream` is.  psi_out equals
 * btmg_mg_cycle's result bit for bit.  Errors as btmg_mg_cycle;
 * BTMG_ERR_OOM if the device buffers cannot be allocated.                 */
int btmg_mg_cycle_host(btmg_problem* p, const void* psi_in, void* psi_out, double* rel_resid, void* stream);

/* Fixed-source solve from the caller's psi: groups in order, each cycled
 * until its relative residual is below rtol or max_cycles; repeated over
 * groups while upscatter makes the all-group residual exceed rtol.  Cycles
 * are replayed from a captured CUDA graph.  Synchronises the stream.
 * info (nullable) receives cycles, final residual and status; the return
 * value is BTMG_OK, or BTMG_ERR_NOT_CONVERGED / _DIVERGED (> 1e3 growth) /
 * _NAN when the iteration failed (psi then holds the last iterate).        */
int btmg_solve(btmg_problem* p, void* psi, double rtol, int32_t max_cycles,
               btmg_solve_info* info, void* stream);

/* Mixed-precision solve with FP64 iterative refinement.  psi64 is a
 * caller-owned device FP64 buffer [G][nd][ny][nx] (initial guess in, solution
 * out).  Each outer step computes r = b - A psi64 in FP64 on the GPU (an
 * internal FP64 copy of the problem), solves the correction equation
 * A delta = r / rms(r) with `inner_cycles` sawtooth cycles whose psi is
 * stored in the problem's psi_dtype (BF16/FP16/FP32, FP32 accumulation), and
 * adds rms(r) delta to psi64.  Stops when ||r||_W/||q||_W <= rtol or after
 * max_outer corrections.  Needs pg = 0 (the correction equation of the
 * nonlinear PG operator is not this linear one): BTMG_ERR_UNSUPPORTED
 * otherwise.  info->history (optional) receives the FP64 residual of every
 * outer step; info->cycles the inner cycles.  Synchronises the stream.
 * The first call allocates the FP64 copy and three full-size workspaces.   */
int btmg_solve_refined(btmg_problem* p, double* psi64, double rtol, int32_t max_outer,
                       int32_t inner_cycles, btmg_solve_info* info, void* stream);

/* ---- Learned correction: U-net (no counterpart in the paper's solver;
 * the paper's "U-net" is the multigrid cycle itself with fixed weights).
 * A small U-net (4 levels, 16/32/48/64 channels, 3x3 convolutions, average
 * pooling, nearest upsampling with skip concatenation; 196k parameters) run
 * and trained by the library's own BF16 kernels (tensor-core implicit-GEMM
 * convolutions, FP32 accumulation, FP32 master weights, Adam).
 * Inputs are device FP32 [N][H][W][in_channels] (H, W multiples of 8),
 * outputs device FP32 [N][H][W].  Parameters are one flat FP32 vector:
 * per layer weights [cout][ks][ks][cin] then biases [cout].               */
typedef struct btmg_unet btmg_unet;
int btmg_unet_create(int32_t in_channels, uint64_t seed, btmg_unet** out);
int btmg_unet_destroy(btmg_unet* u);
int btmg_unet_num_params(const btmg_unet* u, int64_t* n);
int btmg_unet_get_params(const btmg_unet* u, float* host, int64_t n);
int btmg_unet_set_params(btmg_unet* u, const float* host, int64_t n);
int btmg_unet_get_grads(const btmg_unet* u, float* host, int64_t n);
int btmg_unet_forward(btmg_unet* u, const float* x, float* y, int32_t n, int32_t h, int32_t w, void* stream);
/* One Adam step on the mean squared error against target [N][H][W]
 * (lr = 0: gradients only).  loss (nullable, host) receives the loss before
 * the step; when non-NULL the call synchronises the stream.               */
int btmg_unet_train_step(btmg_unet* u, const float* x, const float* target, int32_t n, int32_t h, int32_t w,
                         float lr, double* loss, void* stream);
const char* btmg_unet_last_error(void);

/* Attach a trained U-net as a learned correction (NULL detaches); the
 * paper's U-net has fixed weights, the learned step is an extension.  It
 * runs in every `every`-th cycle of btmg_solve, btmg_mg_cycle and the inner
 * cycles of btmg_solve_refined.  Such a cycle of group g:
 *   1. phi0 = scalar flux of psi; psi' = the plain cycle of psi;
 *   2. r' = residual of psi', rho' = sum_n p_n r'_n;
 *   3. the U-net (4 input channels, see btmg_learn_features) predicts, on
 *      the coarse canvas (btmg_learn_canvas), the shape e of the scalar-flux
 *      error of psi' from rho', the materials and phi(psi') - phi0; e is
 *      interpolated bilinearly to the nodes and
 *      c_n = (e - (mu_n de/dx + nu_n de/dy) / max(sigma_t, 1/L)) / (4 pi),
 *      the P1 angular flux of e (L = max(lx, ly));
 *   4. c' = M c, the plain cycle applied to c with zero external source;
 *   5. rc = residual of c' (= -L c');
 *   6. psi' += alpha c' with alpha = -<r', rc>_W / <rc, rc>_W (W = p_n dx dy),
 *      the minimiser of the residual norm of psi' + alpha c'; alpha = 0 when
 *      undefined or when the predicted reduction of ||r'||^2 is below 1e-4;
 *      |alpha| rms(phi(c')) <= 1e3 rms(phi(psi') - phi0).
 * The step cannot raise the residual norm of the linear (pg = 0) operator;
 * alpha = 0 is the plain cycle (plain multigrid is the fallback and the
 * arbiter).  Everything runs on the device and solves capture cycles with and
 * without the step as CUDA graphs.  The U-net must outlive its use.
 * Errors: INVALID_ARG (null problem, every < 1), OOM.                      */
int btmg_set_learned(btmg_problem* p, btmg_unet* unet, int32_t every);
/* Particle balance of psi per group for the upwind fine scheme (pg = 0),
 * whose streaming term telescopes over rows and columns so that a converged
 * solution balances to its residual level: out[4 g + 0] production
 * dxdy sum (4 pi s_g + sum_{h != g} sigma_s[g<-h] phi_h), out[4 g + 1]
 * removal dxdy sum (sigma_t,g - sigma_s[g<-g]) phi_g, out[4 g + 2] net
 * leakage through the boundary (outgoing boundary values minus the
 * incoming halo values of Sec. 2.3, weighted p_n |mu_n| dy and
 * p_n |nu_n| dx), out[4 g + 3] (production - removal - leakage) /
 * production.  psi: device [G][nd][ny][nx] of psi_dtype; out: host array
 * of 4 G doubles; FP64 accumulation.  Synchronises the stream.
 * Errors: INVALID_ARG (NULL argument), UNSUPPORTED (pg = 1), CUDA.         */
int btmg_particle_balance(btmg_problem* p, const void* psi, double* out, void* stream);

/* The ConvFEM 1D stencils of an order (Sec. 2.7 and the Appendix) as the
 * library derives them: m1 (mass over lumped mass), d1 (advection) and s1
 * (stiffness) at offsets -3..3 (host arrays of 7; taps beyond the order's
 * half width are 0), h = 1.  Host-only (no device needed).
 * Errors: INVALID_ARG (order outside 1..3, NULL output).                   */
int btmg_convfem_stencils(int32_t order, double* m1, double* d1, double* s1);

/* Number of solves on p that dropped the scattering smoother
 * (desc.scat_levels) for the rest of the call: plain multigrid arbitrates it as
 * it arbitrates the learned step, btmg_solve when a residual exceeds twice its
 * best so far, btmg_solve_refined when an outer FP64 residual exceeds 1.5
 * times its best; the next call starts with the smoother again.  Batched
 * solves do not fall back.  Errors: INVALID_ARG (NULL argument).          */
int btmg_scatter_fallbacks(const btmg_problem* p, int32_t* fallbacks);

/* Learned steps since btmg_set_learned, their mean residual reduction
 * factor ||r' + alpha rc|| / ||r'||, the last alpha, and the number of solves
 * that fell back to plain cycles (synchronises the device).  A solve falls
 * back, for the rest of that call, when its residual exceeds twice its best
 * so far (btmg_solve) or its outer FP64 residual exceeds 1.5 times its best
 * (btmg_solve_refined).
 * Any output may be NULL.                                                   */
int btmg_learn_stats(btmg_problem* p, int64_t* steps, double* mean_factor, double* last_alpha,
                     int32_t* fallbacks);
/* Coarse canvas of the learned correction: factor f = ceil(max(nx, ny) / 64)
 * and the canvas ceil(ny / f) x ceil(nx / f), each rounded up to a multiple
 * of 8; canvas pixel (X, Y) covers the nodes [X f, X f + f) x [Y f, Y f + f). */
int btmg_learn_canvas(const btmg_problem* p, int32_t* h8, int32_t* w8, int32_t* factor);
/* Features of the learned step for psi (training pairs): feat device FP32
 * [G][H8][W8][4] on the coarse canvas, each pixel the mean over its nodes:
 * (rho / rms(rho), log(sigma_t f dx + 1e-3) / 4 with the mean sigma_t,
 * mean sigma_s / mean sigma_t, dphi / rms(dphi)) with rho = sum_n p_n r_n of
 * the residual of psi and dphi = phi - phi_prev, the change of scalar flux
 * from psi_prev to psi (psi_prev nullable: channel 3 = 0); the rms are over
 * the covered canvas pixels; zero outside them.  scale device FP32 [G] =
 * rms of the mean rho of each group.                                       */
int btmg_learn_features(btmg_problem* p, const void* psi, const void* psi_prev, float* feat, float* scale,
                        void* stream);

/* Measurement helper (no counterpart in the paper): the FP32 FMA rate of
 * this GPU in TFLOP/s, the best of `repeats` (>= 1) timed launches (after one
 * warm-up) of a kernel that runs 8 independent fmaf chains per thread on
 * every SM at full occupancy; CUDA events on `stream`.  Used beside the
 * ALU roofline peak derived from unit counts and clock.
 * Errors: INVALID_ARG, OOM, CUDA.                                          */
int btmg_fp32_fma_rate(int32_t repeats, double* tflops, void* stream);

/* Failure-path self-test (no counterpart in the paper).  Every wait of the
 * staged kernels on a copy (mbarrier) is bounded: when it gives up the kernel
 * sets the problem's error flag, drains its copies and returns, and the next
 * call that reads the flag returns BTMG_ERR_TIMEOUT with the context still
 * usable.  This call runs that path on purpose: a kernel waits, with `polls`
 * polls (>= 1), on an mbarrier that nothing arrives on.  Returns
 * BTMG_ERR_TIMEOUT (the expected outcome), INVALID_ARG or CUDA.            */
int btmg_wait_selftest(int32_t polls, void* stream);

/* ------------------------------------------------------------------------
 * Batched solves of independent problems (no counterpart in the paper: its
 * solver treats one problem at a time).
 *
 * btmg_create_batch creates n problems from descs[0..n-1] (each as
 * btmg_create_problem).  With autotune = 1, the direction-chunk count of
 * every distinct problem shape (nx, ny, directions, groups, psi_dtype, pg,
 * nu_jacobi) is chosen by timing: each candidate divisor of the direction
 * count (at most 64, within a factor 4 of the automatic choice) runs 2
 * warm-up and 3 timed eager cycles on a scratch copy of the problem (CUDA
 * events on `stream`); the fastest is kept.  Choices are cached per shape
 * for the life of the process.  descs[i].chunks != 0 is kept as given.
 *
 * btmg_solve_batch solves every problem i from its caller-owned device
 * psi[i] (layout of btmg_get_layout; initial guess in, solution out): one
 * eager cycle per problem, then one CUDA graph advances every unconverged
 * problem by a cycle.  When every problem has one group, FP32 compute
 * (FP32/BF16/FP16 storage), no scattering smoother and the same nu <= 4, the
 * graph holds each problem's fine residual (with its source and norm), then
 * ONE persistent launch that does the coarse correction of all of them (the
 * restrictions down every level and the nu upwind Jacobi sweeps from the
 * coarsest level up to level 1, Sec. 2.5): its CTAs drain a device queue of
 * (problem, level, block) tasks, each waiting, bounded by about a second, for
 * the previous level of its problem to complete (a wait that gives up makes
 * the call return BTMG_ERR_TIMEOUT), then each problem's finest sweeps and
 * PG Jacobi.  With autotune = 1 the persistent launch's sweep tile width (16
 * or 32 nodes) and grid (1, 2 or 4 CTAs per SM) are chosen by timing 5
 * launches of each on the first cycle's residuals (CUDA events).  Other
 * batches hold each problem's whole cycle as an independent branch.  The
 * graph also copies the residual norms to the host.  Every check_every
 * launches the residuals are read; converged, failed or exhausted problems
 * leave the graph, which is then rebuilt.  infos[i] (nullable array, history
 * ignored) receives cycles, status and the FP64 relative residual of the
 * returned psi as btmg_solve.  Returns BTMG_OK when every problem
 * converged, else BTMG_ERR_NOT_CONVERGED (or the first hard error).  Learned
 * corrections are not applied in batched solves.
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT (a bounded device wait gave up).  */
typedef struct btmg_batch btmg_batch;
int btmg_create_batch(const btmg_problem_desc* descs, int32_t n, int32_t autotune, void* stream,
                      btmg_batch** out);
int btmg_destroy_batch(btmg_batch* b);
/* Problem i of the batch (owned by the batch; do not destroy it).         */
int btmg_batch_problem(btmg_batch* b, int32_t i, btmg_problem** p);
/* Chunk count of problem i, the automatic choice for its shape, and the
 * tuned time of one eager cycle in ms (0 when not tuned).                  */
int btmg_batch_chunks(const btmg_batch* b, int32_t i, int32_t* chunks, int32_t* auto_chunks, double* ms);
/* Whether the batch's coarse corrections run in the persistent launch, its
 * sweep tile width, CTAs per SM, and the tuned time of one launch in ms (0
 * before tuning or without autotune).  Any output may be NULL.            */
int btmg_batch_coarse(const btmg_batch* b, int32_t* persistent, int32_t* tile, int32_t* ctas, double* ms);
/* Failure-path self-test of the persistent launch (no counterpart in the
 * paper): a queue of one task whose prerequisite never completes; its wait
 * gives up after about a second, sets the launch's error word and the CTA
 * ends.  Returns BTMG_ERR_TIMEOUT (the expected outcome), OOM or CUDA.    */
int btmg_batch_wait_selftest(void* stream);
int btmg_solve_batch(btmg_batch* b, void* const* psi, double rtol, int32_t max_cycles, int32_t check_every,
                     btmg_solve_info* infos, void* stream);

/* Instrumentation (no counterpart in the paper; used by the benchmark).
 * btmg_profile(p, 1) brackets every subsequent kernel launch of the cycle
 * with two CUDA events on the launching stream; btmg_profile_read()
 * synchronises on them and returns, per kernel class, the summed device
 * milliseconds and the number of launches, then clears the record.
 * Classes: 0 PG residual, 1 PG Jacobi, 2 finest-level upwind Jacobi+update,
 * 3 coarse upwind Jacobi, 4 restriction, 5 scalar flux / source / sums.
 * Launches made while capturing the solve graph are not bracketed.
 * btmg_launch_count() returns the number of kernels this problem has
 * launched (replays of a captured graph are not counted).                  */
#define BTMG_PROF_CLASSES 6
int btmg_profile(btmg_problem* p, int32_t enable);
int btmg_profile_read(btmg_problem* p, double* ms, int64_t* count, int32_t n_classes);
int btmg_launch_count(const btmg_problem* p, int64_t* n);

/* Allocation-free residual (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory: a host program or
 * framework that reserves the GPU's memory up front for its own pool and
 * gives every library a fixed budget (an allocation inside the library would
 * fail or fragment that pool), a latency-critical loop in which cudaMalloc
 * and cudaFree, which may synchronise the device, are not acceptable, or an
 * embedded runtime that lends no device allocator to libraries.  It computes
 * what btmg_apply_operator computes for one group in FP32,
 * r = b - A psi with b = s + sigma_s phi / (4 pi), without a problem handle
 * and without allocating: it calls no cudaMalloc, cudaFree or allocating
 * routine and copies no host memory to the device.  Its scratch (scalar
 * flux, source, direction table, error word, norm partial sums) is one
 * file-scope device array of BTMG_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits.
 *   nx, ny, lx, ly, n_polar, n_azim, bc, pg, pg_half: as in btmg_problem_desc
 *     (quadratic ConvFEM; nx*ny <= BTMG_NOALLOC_MAX_NODES and
 *     8*(n_polar/2)*(n_azim/4) <= BTMG_NOALLOC_MAX_DIRS, and the norm
 *     partial sums of the residual kernel must fit the scratch (very thin
 *     grids with pg = 0 do not); otherwise BTMG_ERR_NOALLOC_TOO_LARGE is
 *     returned and nothing is launched);
 *   sigma_t, sigma_s, source: caller-owned device float arrays [ny][nx]
 *     (total, in-group isotropic scattering, isotropic source per node);
 *   psi: caller-owned device float [nd][ny][nx]; r: same shape, output;
 *   rel_resid: nullable host pointer.  NULL: the call only enqueues its
 *     kernels on `stream` and returns.  Non-NULL: it also reduces the norms,
 *     synchronises `stream`, stores ||r||_W / ||s||_W (W = p_n dx dy, FP64
 *     sums) and returns BTMG_ERR_TIMEOUT if a bounded wait of the residual
 *     kernel gave up, in which case r is incomplete.  Only a call with
 *     rel_resid reports such a timeout; the error word is cleared at the
 *     start of every call.
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call reuses the same scratch and leaves its contents
 * behind; each call writes all scratch it reads before reading it, so none
 * needs clearing, but calls that overlap on the GPU (concurrent streams)
 * race on it.                                                              */
#define BTMG_NOALLOC_MAX_NODES (512 * 512)
#define BTMG_NOALLOC_MAX_DIRS 2048
#define BTMG_NOALLOC_SCRATCH_BYTES (2359296)
#define BTMG_ERR_NOALLOC_TOO_LARGE (-9)
int btmg_apply_operator_noalloc(int32_t nx, int32_t ny, double lx, double ly, int32_t n_polar,
                                int32_t n_azim, const int32_t bc[4], int32_t pg, int32_t pg_half,
                                const float* sigma_t, const float* sigma_s, const float* source,
                                const float* psi, float* r, void* stream, double* rel_resid);

const char* btmg_error_string(int status);
const char* btmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BTMG_H */
