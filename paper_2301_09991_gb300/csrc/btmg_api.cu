// btmg_api.cu -- host side of the btmg C ABI: problem set-up (octahedral
// quadrature of Sec. 2.2, space-angle hierarchy of Sec. 2.5), device
// workspaces, the sawtooth cycle sequencing of Fig. multi_grid_it and the
// CUDA-graph solve loop.  Every arithmetic step of the iteration runs in the
// kernels of k_pg.cu and k_mg.cu; the host only launches them.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/btmg.h"
#include "btmg_common.cuh"

using namespace btmg;

int unet_in_channels(const btmg_unet* u);  // defined with the U-net kernels

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CK(...)                                                                                       \
  do {                                                                                                \
    cudaError_t e_ = (__VA_ARGS__);                                                                   \
    if (e_ != cudaSuccess)                                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? BTMG_ERR_OOM : BTMG_ERR_CUDA,                     \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr int kTile = 32;  // tile edge of the PG and upwind kernels
constexpr int kOutParts = 4;  // direction ranges of the host-buffer cycle's final launch
// multiprocessors of the current device (152 on GB300 if the query fails)
int device_sms() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}
constexpr int kDotBlocks = 4 * 152;  // blocks of the learned-step dot product (4 per SM)

// ------------------------------------------------- quadrature (Sec. 2.2) --
// Gauss-Legendre on [0,1]: Newton iteration on the three-term recurrence.
void gauss_legendre_unit(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double t = std::cos(kPi * (4.0 * k + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pm = 0.0, p = 1.0;
      for (int m = 1; m <= n; ++m) {
        const double pn = ((2.0 * m - 1.0) * t * p - (m - 1.0) * pm) / m;
        pm = p;
        p = pn;
      }
      dp = n * (pm - t * p) / (1.0 - t * t);
      const double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[k] = 0.5 * (1.0 + t);
    w[k] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Directions of the 8 octahedron faces, each with an nr x nc grid mapped by
// X(u,t) = (1-t)((1-u) a + u b) + t c (corners a, b, c on the axes, the edge
// t = 1 collapsed onto c) and projected radially onto the unit sphere.  The
// solid angle element of the projection is (X . (X_u x X_t)) / |X|^3 du dt
// = (1-t) / |X|^3 du dt; p_n is its integral over the patch, (mu_n, nu_n)
// the patch-mean direction.  Weights are scaled so that sum p = 4 pi.
void octahedral_quadrature(int nr, int nc, std::vector<double>& mu, std::vector<double>& nu,
                           std::vector<double>& p) {
  const int nd = 8 * nr * nc, ng = 16;
  std::vector<double> gx, gw;
  gauss_legendre_unit(ng, gx, gw);
  mu.assign(nd, 0.0);
  nu.assign(nd, 0.0);
  p.assign(nd, 0.0);
  double total = 0.0;
  for (int f = 0; f < 8; ++f) {
    const double sx = (f & 1) ? -1 : 1, sy = (f & 2) ? -1 : 1, sz = (f & 4) ? -1 : 1;
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < nc; ++i) {
        double area = 0, mx = 0, my = 0;
        for (int a = 0; a < ng; ++a)
          for (int b = 0; b < ng; ++b) {
            const double t = (j + gx[a]) / nr, u = (i + gx[b]) / nc;
            const double X0 = (1 - t) * (1 - u) * sx, X1 = (1 - t) * u * sy, X2 = t * sz;
            const double r2 = X0 * X0 + X1 * X1 + X2 * X2, r = std::sqrt(r2);
            const double dS = gw[a] * gw[b] / (double(nr) * nc) * (1 - t) / (r2 * r);
            area += dS;
            mx += dS * X0 / r;
            my += dS * X1 / r;
          }
        const int n = f * nr * nc + j * nc + i;
        p[n] = area;
        mu[n] = mx / area;
        nu[n] = my / area;
        total += area;
      }
  }
  for (int n = 0; n < nd; ++n) p[n] *= 4.0 * kPi / total;
}

// ConvFEM 1D stencils of order p (Sec. 2.7 and the Appendix), h = 1, stored
// at offsets -3..3 (zero beyond -p..p): the Lagrange element of order p on [0, p] with nodes 0..p gives the
// mass, advection and stiffness matrices M_ab = int N_a N_b,
// C_ab = int N_a N_b', K_ab = int N_a' N_b'; the assembled rows of the p
// node types (the corner, shared by two elements, and the p - 1 interior
// nodes) are averaged and divided by the lumped mass.  The basis functions
// are expanded into monomial coefficients and the products integrated
// exactly (int_0^p x^k dx = p^(k+1) / (k+1)).
void convfem_stencils(int p, double* m1, double* d1, double* s1) {
  double N[4][4] = {}, D[4][4] = {};  // coefficient of x^k of N_a and of N_a'
  for (int a = 0; a <= p; ++a) {
    double c[4] = {1.0, 0.0, 0.0, 0.0};  // prod_{m != a} (x - m) / (a - m)
    int deg = 0;
    for (int m = 0; m <= p; ++m) {
      if (m == a) continue;
      double nc[4] = {};
      for (int k = 0; k <= deg; ++k) {
        nc[k + 1] += c[k] / (a - m);
        nc[k] -= c[k] * m / (a - m);
      }
      ++deg;
      for (int k = 0; k < 4; ++k) c[k] = nc[k];
    }
    for (int k = 0; k <= p; ++k) N[a][k] = c[k];
    for (int k = 1; k <= p; ++k) D[a][k - 1] = k * c[k];
  }
  auto integ = [p](const double* f, const double* g) {  // int_0^p f g, both of degree <= 3
    double s = 0.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (f[i] != 0.0 && g[j] != 0.0) s += f[i] * g[j] * std::pow((double)p, i + j + 1) / (i + j + 1);
    return s;
  };
  double am[7] = {}, ac[7] = {}, ak[7] = {};
  auto add_row = [&](int a, int self) {  // row of local node a; the node sits at local index self
    for (int b = 0; b <= p; ++b) {
      am[b - self + p] += integ(N[a], N[b]);
      ac[b - self + p] += integ(N[a], D[b]);
      ak[b - self + p] += integ(D[a], D[b]);
    }
  };
  add_row(p, p);  // corner: last node of the left element ...
  add_row(0, 0);  // ... and first node of the right one
  for (int k = 1; k < p; ++k) add_row(k, k);
  double mL = 0.0;
  for (int o = 0; o <= 2 * p; ++o) mL += am[o] / p;
  for (int o = 0; o < 7; ++o) m1[o] = d1[o] = s1[o] = 0.0;
  for (int o = 0; o <= 2 * p; ++o) {  // stored at offsets -3..3
    m1[o + 3 - p] = am[o] / p / mL;
    d1[o + 3 - p] = ac[o] / p / mL;
    s1[o + 3 - p] = ak[o] / p / mL;
  }
}

struct LevelH {
  int nx, ny, nr, nc, nd;
  double dx, dy;
  std::vector<double> mu, nu, p;
  std::vector<double> sig;  // [G][ny][nx]
  int fx = 1, fy = 1, fr = 1, fc = 1;  // factors to the next coarser level
  size_t npix() const { return (size_t)nx * ny; }
  size_t n() const { return (size_t)nd * nx * ny; }
};

size_t dtype_size(int t) { return t == BTMG_F64 ? 8 : t == BTMG_F32 ? 4 : 2; }

}  // namespace

struct btmg_problem {
  btmg_problem_desc d{};
  int G = 0, L = 0, dtype = BTMG_F32;
  bool f64 = false;
  size_t csize = 4;  // compute element size
  std::vector<LevelH> lev;
  int dpc = 1, nchunk = 1, tiles_x = 1, tiles_y = 1;
  bool upscatter = false;
  // device buffers (compute type unless noted)
  std::vector<void*> d_dir, d_rcoef, d_sig, d_s, d_delta, d_parent;
  // scattering smoother (desc.scat_levels): per level on/off and gain w
  // [G][npix]; shared sweep scratch (largest smoothed level)
  std::vector<char> scat_on;
  std::vector<void*> d_scat_w;
  void* d_scat_j = nullptr;     // [nd][ny][nx]
  void* d_scat_part = nullptr;  // [chunks][ny][nx]
  void* d_scat_c = nullptr;     // [ny][nx]
  int scat_tail = 0;            // first level of the smoother's single-CTA tail (L: none)
  int plain_tail = 0;           // first level of the published cycle's single-CTA tail
  bool scat_off = false;        // solve-time fallback to the plain sweeps
  double st_m1[7] = {}, st_d1[7] = {}, st_s1[7] = {};  // ConvFEM 1D stencils of the order
  void* d_pgd = nullptr;        // cubic PG scratch: Psi_x, Psi_y, k_x, k_y [4][nd][ny][nx]
  int32_t scat_fallbacks = 0;   // solves that fell back
  void* d_sigs = nullptr;      // [G][G][npix]
  void* d_src = nullptr;       // [G][npix]
  void* d_b = nullptr;         // [npix]
  void* d_phi_part = nullptr;  // [G][nchunk][npix]
  void* d_psi_tmp = nullptr;   // storage type, one group
  double* d_norm_part = nullptr;
  int n_norm_part = 0;  // allocated norm partials
  int n_norm_sum = 0;   // norm partials written by the fine residual kernel
  double* d_qn2_part = nullptr;
  int n_q_blocks = 0;
  double* d_rn2 = nullptr;  // [G]
  double* d_qn2 = nullptr;  // [G]
  double* h_pinned = nullptr;  // [2G + 1]
  int* d_err = nullptr;        // device error word (bounded waits)
  // captured cycle graphs per group
  std::vector<cudaGraphExec_t> graphs;   // plain cycle
  std::vector<cudaGraphExec_t> lgraphs;  // cycle with the learned step
  const void* graph_psi = nullptr;
  cudaStream_t graph_stream = nullptr;
  // graphs cannot be captured on the legacy default stream: solve() runs on
  // this stream when the caller passes NULL, ordered after the caller's work
  cudaStream_t own_stream = nullptr;
  cudaEvent_t order_event = nullptr;
  // host copies of the problem statement (to build the FP64 twin)
  std::vector<int32_t> h_region;
  std::vector<double> h_sigma_t, h_sigma_s, h_source;
  // iterative refinement: FP64 twin (residuals), correction workspaces
  btmg_problem* twin = nullptr;
  void* d_zero_src = nullptr;       // [G][npix] zeros (compute type)
  const void* inner_extra = nullptr;  // [G][nd][ny][nx] anisotropic source or NULL
  bool zero_src = false;
  void* d_delta_all = nullptr;      // [G][nd][ny][nx] storage type
  void* d_extra_all = nullptr;      // [G][nd][ny][nx] compute type
  double* d_r64 = nullptr;          // [G][nd][ny][nx]
  // learned correction (btmg_set_learned)
  btmg_unet* learned = nullptr;
  int learn_every = 1;
  int H8 = 8, W8 = 8, lf = 1;  // coarse canvas of the learned correction and its factor
  void* d_rho_part = nullptr;   // [G][nchunk][npix] compute type
  float* d_feat = nullptr;      // [H8][W8][3]
  float* d_dimg = nullptr;      // [H8][W8]
  float* d_lscale = nullptr;    // [1]
  double* d_lsum = nullptr;
  double* d_lpart = nullptr;    // [max(2 kLearnBlocks, n_q_blocks)]
  void* d_lc = nullptr;         // [nd][ny][nx] P1 correction c (storage type)
  void* d_lr = nullptr;         // [nd][ny][nx] residual of c, -L c (compute type)
  void* d_lb = nullptr;         // [ny][nx] scattering source of c (compute type)
  double* d_ldot = nullptr;     // [2] <r1, rc>, <rc, rc>
  double* d_ldpart = nullptr;   // [kDotBlocks]
  double* d_lstat = nullptr;    // [3] sum of residual reduction factors, steps, last alpha
  void* d_lphi = nullptr;       // [nchunk][ny][nx] scalar-flux partials of c (compute type)
  void* d_lzero = nullptr;      // [ny][nx] zeros (compute type)
  void* d_lphi0 = nullptr;      // [ny][nx] scalar flux before the cycle (compute type)
  void* d_lprev_all = nullptr;  // [G][ny][nx] scalar flux of psi_prev (btmg_learn_features)
  int64_t learn_count = 0;      // mg_cycle calls since the net was attached
  bool learn_off = false;       // solve-time fallback to plain cycles (reset by each solve)
  int32_t learn_fallbacks = 0;  // solves that fell back since the net was attached
  // host-buffer cycle (btmg_mg_cycle_host): device copy of psi, and while a
  // call runs the host destination of every group's final PG Jacobi, which
  // is streamed out in direction ranges on the side streams
  void* d_hpsi = nullptr;  // [G][nd][ny][nx] storage type
  void* d_hzero = nullptr; // [ny][nx] zeros (compute type): the source of the range residuals
  double* d_hparts = nullptr;  // residual-norm partials of the level-1 restriction that forms r
  int n_hparts = 0;
  bool first_restricted = false;  // level 1's source is already formed (skip the first restriction)
  void* out_host = nullptr;
  cudaStream_t out_s[kOutParts] = {};
  cudaEvent_t out_ev[kOutParts + 1] = {};
  // per-kernel-class CUDA-event timing (btmg_profile) and launch counting
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<int> prof_cls;
  int64_t launches = 0;
};

namespace {

template <typename C> C* dptr(void* p) { return reinterpret_cast<C*>(p); }

void free_graphs(btmg_problem* P) {
  for (auto* v : {&P->graphs, &P->lgraphs}) {
    for (auto& g : *v)
      if (g) cudaGraphExecDestroy(g);
    v->assign(P->G, nullptr);
  }
  P->graph_psi = nullptr;
}

void destroy(btmg_problem* P);
int create(const btmg_problem_desc* d, btmg_problem** out);

// --------------------------------------------------------------- launches --
// Kernel classes reported by btmg_profile_read (BTMG_PROF_*).
enum { PC_PG_RESID = 0, PC_PG_JACOBI = 1, PC_UP_FINE = 2, PC_UP_COARSE = 3, PC_RESTRICT = 4, PC_MISC = 5, PC_N = 6 };

// Launches f() on stream s; counts the launch and, when profiling, brackets
// it with two CUDA events recorded on the same stream.
template <class F> cudaError_t timed(btmg_problem* P, int cls, cudaStream_t s, F&& f) {
  ++P->launches;
  if (!P->prof_on) return f();
  const size_t k = 2 * P->prof_cls.size();
  while (P->prof_pool.size() < k + 2) {
    cudaEvent_t e;
    cudaError_t ec = cudaEventCreate(&e);
    if (ec != cudaSuccess) return ec;
    P->prof_pool.push_back(e);
  }
  cudaError_t e0 = cudaEventRecord(P->prof_pool[k], s);
  if (e0 != cudaSuccess) return e0;
  cudaError_t e = f();
  if (e != cudaSuccess) return e;
  P->prof_cls.push_back(cls);
  return cudaEventRecord(P->prof_pool[k + 1], s);
}

template <typename T, typename C> struct Impl {
  static PgArgs<T, C> pg_args(btmg_problem* P, int g, const T* psi) {
    const LevelH& L0 = P->lev[0];
    PgArgs<T, C> a{};
    a.psi = psi;
    a.b = dptr<C>(P->d_b);
    a.sigt = dptr<C>(P->d_sig[0]) + (size_t)g * L0.npix();
    a.dir = reinterpret_cast<const Dir<C>*>(P->d_dir[0]);
    a.nx = L0.nx;
    a.ny = L0.ny;
    a.nd = L0.nd;
    a.dpc = P->dpc;
    a.tiles_x = P->tiles_x;
    a.dx = (C)L0.dx;
    a.dy = (C)L0.dy;
    a.inv_dx = (C)(1.0 / L0.dx);
    a.inv_dy = (C)(1.0 / L0.dy);
    a.inv_dx2 = (C)(1.0 / (L0.dx * L0.dx));
    a.inv_dy2 = (C)(1.0 / (L0.dy * L0.dy));
    a.dxdy = (C)(L0.dx * L0.dy);
    // Sec. 2.6 constants for order p: eps_k = 1e-3, alpha_kabs = 2^p/16,
    // alpha_ksquare = 2^p/2; alpha_r = beta_r = 3.
    a.eps_k = (C)1e-3;
    a.a_kabs = (C)(std::ldexp(1.0, P->d.order) / 16.0);  // 2^p / 16
    a.a_ksq = (C)(std::ldexp(1.0, P->d.order) / 2.0);    // 2^p / 2
    a.order = P->d.order;
    if (P->d.order == 3) {  // the cubic path's stencils (offsets -3..3) and scratch
      for (int o = 0; o < 7; ++o) {
        a.cm1[o] = (C)P->st_m1[o];
        a.cd1[o] = (C)P->st_d1[o];
        a.cs1[o] = (C)P->st_s1[o];
      }
      const size_t n = L0.n();
      C* base = dptr<C>(P->d_pgd);
      a.gpx = base;
      a.gpy = base + n;
      a.gkx = base + 2 * n;
      a.gky = base + 3 * n;
    }
    a.a_r = (C)3.0;
    a.half = (C)(P->d.pg_half ? 0.5 : 1.0);
    a.beta = (C)(P->d.pg ? P->d.beta_pg : 1.0);
    a.bc = Bc{P->d.bc[0], P->d.bc[1], P->d.bc[2], P->d.bc[3]};
    a.err = P->d_err;
    a.extra = P->inner_extra ? reinterpret_cast<const C*>(P->inner_extra) + (size_t)g * L0.n() : nullptr;
    a.rho_part = nullptr;
    return a;
  }

  // b for group g from the scalar-flux partials of every group; with
  // want_norm the squared norm of its fixed part (external source and the
  // other groups' scattering) lands in d_qn2[g] for the relative residual.
  // want_norm: q's norm partials; sum_norm: also their sum into d_qn2 (else
  // the caller sums them with another reduction)
  static cudaError_t source(btmg_problem* P, int g, cudaStream_t s, bool want_norm = true, bool sum_norm = true) {
    const size_t npix = P->lev[0].npix();
    cudaError_t e = timed(P, PC_MISC, s, [&] {
      const C* src = P->zero_src ? dptr<C>(P->d_zero_src) : dptr<C>(P->d_src);
      return launch_source<C>(src + g * npix, dptr<C>(P->d_sigs) + (size_t)g * P->G * npix,
                              dptr<C>(P->d_phi_part), P->G, g, P->nchunk, (int)npix, dptr<C>(P->d_b), nullptr,
                              want_norm ? P->d_qn2_part : nullptr, P->n_q_blocks, s);
    });
    if (e != cudaSuccess || !want_norm || !sum_norm) return e;
    return timed(P, PC_MISC, s, [&] { return launch_sum(P->d_qn2_part, P->n_q_blocks, P->d_qn2 + g, s); });
  }

  // In-group scattering source of the learned correction from its partials
  // d_lphi: d_lb = (sigma_s,gg / 4 pi) phi_c (no external source).
  static cudaError_t homog_source(btmg_problem* P, int g, cudaStream_t s) {
    const size_t npix = P->lev[0].npix();
    return timed(P, PC_MISC, s, [&] {
      return launch_source<C>(dptr<C>(P->d_lzero), dptr<C>(P->d_sigs) + ((size_t)g * P->G + g) * npix,
                              dptr<C>(P->d_lphi), 1, 0, P->nchunk, (int)npix, dptr<C>(P->d_lb), nullptr, P->d_lpart,
                              P->n_q_blocks, s);
    });
  }

  static cudaError_t phi_partials(btmg_problem* P, const T* psi, cudaStream_t s) {
    const LevelH& L0 = P->lev[0];
    for (int g = 0; g < P->G; ++g) {
      cudaError_t e = timed(P, PC_MISC, s, [&] {
        return launch_phi_partial<T, C>(psi + (size_t)g * L0.n(),
                                        dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * L0.npix(),
                                        reinterpret_cast<const Dir<C>*>(P->d_dir[0]), L0.nx, L0.ny, L0.nd, P->dpc,
                                        P->nchunk, s);
      });
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  static UpArgs<T, C> up_args(btmg_problem* P, int l, int g) {
    const LevelH& A = P->lev[l];
    UpArgs<T, C> u{};
    u.sig = dptr<C>(P->d_sig[l]) + (size_t)g * A.npix();
    u.dir = reinterpret_cast<const Dir<C>*>(P->d_dir[l]);
    u.nx = A.nx;
    u.ny = A.ny;
    u.nr = A.nr;
    u.nc = A.nc;
    u.nd = A.nd;
    u.nu = P->d.nu_jacobi;
    u.src_stride = A.npix();
    u.tiles_x = (A.nx + kTile - 1) / kTile;
    u.bc = Bc{P->d.bc[0], P->d.bc[1], P->d.bc[2], P->d.bc[3]};
    u.dpc = 1;
    u.err = P->d_err;
    if (l + 1 < P->L) {
      const LevelH& B = P->lev[l + 1];
      u.nxc = B.nx;
      u.nyc = B.ny;
      u.nrc = B.nr;
      u.ncc = B.nc;
      u.fx = A.fx;
      u.fy = A.fy;
      u.fr = A.fr;
      u.fc = A.fc;
      u.parent = reinterpret_cast<const int*>(P->d_parent[l]);
    }
    return u;
  }

  // `sweeps` node-block sweeps of the scattering smoother on level l, group
  // g, from the initial correction of init_mode (INIT_ZERO; INIT_UPSAMPLE of
  // d_delta[l + 1]; INIT_SAME of `init`).  The result delta lands in
  // d_delta[l]; with psi_out set (finest level) the final pass writes
  // psi_out = psi_in + delta and the scalar-flux partials of psi_out instead.
  static cudaError_t scat_level(btmg_problem* P, int l, int g, const C* src, int init_mode, const C* init,
                                int sweeps, const T* psi_in, T* psi_out, C* phi_part, int cls, cudaStream_t s) {
    const LevelH& A = P->lev[l];
    const int nch = scat_chunks(A.nx, A.ny, A.nd, (int)P->csize);
    const int dpc = (A.nd + nch - 1) / nch;
    C* X = dptr<C>(P->d_delta[l]);  // the last sweep writes here
    C* Y = dptr<C>(P->d_scat_j);
    const C* w = dptr<C>(P->d_scat_w[l]) + (size_t)g * A.npix();
    const C* sig = dptr<C>(P->d_sig[l]) + (size_t)g * A.npix();
    const Dir<C>* dir = reinterpret_cast<const Dir<C>*>(P->d_dir[l]);
    C* part = dptr<C>(P->d_scat_part);
    C* cf = dptr<C>(P->d_scat_c);
    cudaError_t e;
    const C* prev = init;
    for (int k = 1; k <= sweeps; ++k) {
      ScatArgs<C> a{};
      a.src = src;
      a.src_stride = A.npix();
      a.init_mode = k == 1 ? init_mode : INIT_SAME;
      a.jin = prev;
      a.cin = k == 1 ? nullptr : cf;
      if (k == 1 && init_mode == INIT_UPSAMPLE) {
        const LevelH& B = P->lev[l + 1];
        a.coarse = dptr<C>(P->d_delta[l + 1]);
        a.parent = reinterpret_cast<const int*>(P->d_parent[l]);
        a.nxc = B.nx;
        a.nyc = B.ny;
        a.fx = A.fx;
        a.fy = A.fy;
      }
      a.jout = (sweeps - k) % 2 == 0 ? X : Y;
      a.part = part;
      a.sig = sig;
      a.dir = dir;
      a.nx = A.nx;
      a.ny = A.ny;
      a.nd = A.nd;
      a.dpc = dpc;
      a.bc = Bc{P->d.bc[0], P->d.bc[1], P->d.bc[2], P->d.bc[3]};
      if ((e = timed(P, cls, s, [&] { return launch_scat_sweep<C>(a, nch, s); })) != cudaSuccess) return e;
      if ((e = timed(P, cls, s, [&] { return launch_scat_corr<C>(part, nch, w, (int)A.npix(), cf, s); })) !=
          cudaSuccess)
        return e;
      prev = a.jout;
    }
    ScatFinal<T, C> f{};
    f.j = X;
    f.c = cf;
    f.sig = sig;
    f.dir = dir;
    f.nx = A.nx;
    f.ny = A.ny;
    f.nd = A.nd;
    if (psi_out) {
      f.psi_in = psi_in;
      f.psi_out = psi_out;
      f.phi_part = phi_part;
      f.dpc = P->dpc;
      return timed(P, cls, s, [&] { return launch_scat_final<T, C>(f, P->nchunk, s); });
    }
    f.delta_out = X;
    f.dpc = dpc;
    return timed(P, cls, s, [&] { return launch_scat_final<T, C>(f, nch, s); });
  }

  // One sawtooth cycle of group g (Fig. multi_grid_it); the scalar-flux
  // partials of every group must describe the current psi on entry and
  // describe the updated psi on exit.  Part A evaluates the residual of the
  // input (and its norm, and the residual moment when a learned correction
  // is attached); part B does the rest of the cycle.
  static cudaError_t cycle_part_a(btmg_problem* P, T* psi_g, int g, cudaStream_t s) {
    cudaError_t e;
    const LevelH& L0 = P->lev[0];
    // 1. r_1 = b - A psi  (Eq. Petrov), weighted norm; the source norm is
    // summed with the residual norm in one launch
    if ((e = source(P, g, s, true, false)) != cudaSuccess) return e;
    PgArgs<T, C> a = pg_args(P, g, psi_g);
    a.r_out = dptr<C>(P->d_s[0]);
    a.norm_part = P->d_norm_part;
    if (P->learned) a.rho_part = dptr<C>(P->d_rho_part) + (size_t)g * P->nchunk * L0.npix();
    if ((e = timed(P, PC_PG_RESID, s, [&] { return launch_pg<T, C>(a, PG_RESID, P->d.pg != 0, P->nchunk, s); })) !=
        cudaSuccess)
      return e;
    return timed(P, PC_MISC, s, [&] {
      return launch_sum2(P->d_norm_part, P->n_norm_sum, P->d_rn2 + g, P->d_qn2_part, P->n_q_blocks, P->d_qn2 + g, s);
    });
  }

  // With `homog`, the cycle of the learned correction c (in P->d_lc, its
  // residual in d_s[0]): zero external source, no inner-refinement source,
  // scalar-flux partials in d_lphi, result back in d_lc.
  // coarse_external: the restrictions and the coarse sweeps (steps 2-4) ran
  // elsewhere (the persistent batched launch) and d_delta[1] holds their result
  static cudaError_t cycle_part_b(btmg_problem* P, T* psi_g, int g, cudaStream_t s, bool homog = false,
                                  bool coarse_external = false) {
    cudaError_t e;
    const int L = P->L;
    const LevelH& L0 = P->lev[0];
    if (!coarse_external) {
    // the smallest levels run in one single-CTA launch (restrictions and
    // sweeps): the smoother's levels while it is active, else the
    // published cycle's when the smoother is off
    int tail = L;
    bool tail_scat = false;
    if (P->scat_tail < L && !P->scat_off) {
      tail = P->scat_tail;
      tail_scat = true;
    } else if (P->d.scat_levels == 0 || P->scat_off) {
      tail = P->plain_tail;
    }
    // 2. restriction to every coarser level (those of the tail inside it)
    for (int l = P->first_restricted ? 1 : 0; l + 1 < L && l < tail; ++l) {
      const LevelH &A = P->lev[l], &B = P->lev[l + 1];
      if ((e = timed(P, PC_RESTRICT, s, [&] {
             return launch_restrict<C>(dptr<C>(P->d_s[l]), dptr<C>(P->d_s[l + 1]), dptr<C>(P->d_rcoef[l]), A.nx,
                                       A.ny, A.nr, A.nc, B.nx, B.ny, B.nr, B.nc, A.fx, A.fy, A.fr, A.fc, s);
           })) != cudaSuccess)
        return e;
    }
    // 3./4. upwind Jacobi from the coarsest level up, UpSamp in between
    int top = L - 1;
    if (tail < L) {
      ScatTail<C> t{};
      t.count = L - tail;
      t.nu = P->d.nu_jacobi;
      t.scat = tail_scat ? 1 : 0;
      t.bc = Bc{P->d.bc[0], P->d.bc[1], P->d.bc[2], P->d.bc[3]};
      t.out = dptr<C>(P->d_delta[tail]);
      for (int k = 0; k < t.count; ++k) {
        const int l = tail + k;
        const LevelH& A = P->lev[l];
        ScatTailLevel<C>& v = t.lev[k];
        v.s = dptr<C>(P->d_s[l]);
        v.rcoef = l + 1 < L ? dptr<C>(P->d_rcoef[l]) : nullptr;
        v.w = tail_scat ? dptr<C>(P->d_scat_w[l]) + (size_t)g * A.npix() : nullptr;
        v.sig = dptr<C>(P->d_sig[l]) + (size_t)g * A.npix();
        v.dir = reinterpret_cast<const Dir<C>*>(P->d_dir[l]);
        v.parent = l + 1 < L ? reinterpret_cast<const int*>(P->d_parent[l]) : nullptr;
        v.nx = A.nx;
        v.ny = A.ny;
        v.nr = A.nr;
        v.nc = A.nc;
        v.nd = A.nd;
        v.fx = A.fx;
        v.fy = A.fy;
        v.fr = A.fr;
        v.fc = A.fc;
      }
      if ((e = timed(P, PC_UP_COARSE, s, [&] { return launch_scat_tail<C>(t, s); })) != cudaSuccess) return e;
      top = tail - 1;
    }
    for (int l = top; l >= 1; --l) {
      if (P->scat_on[l] && !P->scat_off) {
        const int im = (l == L - 1) ? INIT_ZERO : INIT_UPSAMPLE;
        if ((e = scat_level(P, l, g, dptr<C>(P->d_s[l]), im, nullptr, P->d.nu_jacobi, nullptr, nullptr, nullptr,
                            PC_UP_COARSE, s)) != cudaSuccess)
          return e;
        continue;
      }
      UpArgs<T, C> u = up_args(P, l, g);
      u.src = dptr<C>(P->d_s[l]);
      u.init_mode = (l == L - 1) ? INIT_ZERO : INIT_UPSAMPLE;
      u.init = (l == L - 1) ? nullptr : dptr<C>(P->d_delta[l + 1]);
      u.delta_out = dptr<C>(P->d_delta[l]);
      // directions per CTA: as many (up to 8) as still leave two waves of
      // CTAs, so that each CTA's next direction is fetched during its sweeps
      const int nd_l = P->lev[l].nd, tiles_l = u.tiles_x * ((P->lev[l].ny + kTile - 1) / kTile);
      int dpc_l = 1;
      while (dpc_l < 8 && nd_l % (2 * dpc_l) == 0 && (long)tiles_l * (nd_l / (2 * dpc_l)) >= 2L * 3 * device_sms()) dpc_l *= 2;
      u.dpc = dpc_l;
      if ((e = timed(P, PC_UP_COARSE, s, [&] { return launch_upwind<T, C>(u, UP_CORR, nd_l / dpc_l, s); })) !=
          cudaSuccess)
        return e;
    }
    }  // !coarse_external
    // 4./5. finest level: nu sweeps from UpSamp(delta_2), psi_tmp = psi + delta
    if (P->scat_on[0] && !P->scat_off) {
      C* ph = homog ? dptr<C>(P->d_lphi) : dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * L0.npix();
      if ((e = scat_level(P, 0, g, dptr<C>(P->d_s[0]), L > 1 ? INIT_UPSAMPLE : INIT_ZERO, nullptr, P->d.nu_jacobi,
                          psi_g, dptr<T>(P->d_psi_tmp), ph, PC_UP_FINE, s)) != cudaSuccess)
        return e;
    } else {
      UpArgs<T, C> u = up_args(P, 0, g);
      u.src = dptr<C>(P->d_s[0]);
      u.init_mode = (L > 1) ? INIT_UPSAMPLE : INIT_ZERO;
      u.init = (L > 1) ? dptr<C>(P->d_delta[1]) : nullptr;
      u.psi_in = psi_g;
      u.psi_out = dptr<T>(P->d_psi_tmp);
      u.phi_part = homog ? dptr<C>(P->d_lphi) : dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * L0.npix();
      u.dpc = P->dpc;
      if ((e = timed(P, PC_UP_FINE, s, [&] { return launch_upwind<T, C>(u, UP_UPDATE, P->nchunk, s); })) !=
          cudaSuccess)
        return e;
    }
    // 6. fine PG Jacobi sweep with diagonal beta d (Eq. matrix_full)
    if ((e = homog ? homog_source(P, g, s) : source(P, g, s, false)) != cudaSuccess) return e;
    PgArgs<T, C> j = pg_args(P, g, dptr<T>(P->d_psi_tmp));
    j.psi_out = psi_g;
    j.phi_part = dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * L0.npix();
    if (homog) {
      j.b = dptr<C>(P->d_lb);
      j.extra = nullptr;
      j.phi_part = dptr<C>(P->d_lphi);
    }
    if (homog || !P->out_host)
      return timed(P, PC_PG_JACOBI, s, [&] { return launch_pg<T, C>(j, PG_JACOBI, P->d.pg != 0, P->nchunk, s); });
    return jacobi_to_host(P, j, g, s);
  }

  // The final PG Jacobi of group g with its result copied to P->out_host.
  // The paired FP32 kernel runs as kOutParts launches over consecutive
  // direction-chunk ranges, each on its own side stream and followed there
  // by the copy of its directions, so the copies of the first ranges overlap
  // the kernels of the later ones (the ranges share no data: each writes its
  // own directions and chunk partials).  Otherwise one launch, then the
  // group's copy on a side stream (it overlaps the next group's cycle).
  // The side streams fork from and join back into s through events.
  static cudaError_t jacobi_to_host(btmg_problem* P, PgArgs<T, C>& j, int g, cudaStream_t s) {
    const LevelH& L0 = P->lev[0];
    const size_t plane = L0.npix() * sizeof(T);
    char* hout = reinterpret_cast<char*>(P->out_host) + (size_t)g * L0.nd * plane;
    const char* dsrc = reinterpret_cast<const char*>(j.psi_out);
    bool split = false;
    if constexpr (std::is_same<T, float>::value && std::is_same<C, float>::value)
      split = P->d.pg != 0 && P->nchunk % kOutParts == 0 && pg2_applies(j);
    cudaError_t e;
    if (!split) {
      if ((e = launch_pg<T, C>(j, PG_JACOBI, P->d.pg != 0, P->nchunk, s)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(P->out_ev[0], s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(P->out_s[0], P->out_ev[0], 0)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(hout, dsrc, L0.nd * plane, cudaMemcpyDeviceToHost, P->out_s[0])) != cudaSuccess)
        return e;
      if ((e = cudaEventRecord(P->out_ev[1], P->out_s[0])) != cudaSuccess) return e;
      return cudaStreamWaitEvent(s, P->out_ev[1], 0);
    }
    if ((e = cudaEventRecord(P->out_ev[0], s)) != cudaSuccess) return e;
    const int per = P->nchunk / kOutParts;
    const size_t bytes = (size_t)per * P->dpc * plane;
    for (int i = 0; i < kOutParts; ++i) {
      cudaStream_t si = P->out_s[i];
      if ((e = cudaStreamWaitEvent(si, P->out_ev[0], 0)) != cudaSuccess) return e;
      PgArgs<T, C> ji = j;
      ji.chunk0 = i * per;
      if ((e = launch_pg<T, C>(ji, PG_JACOBI, true, per, si)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(hout + i * bytes, dsrc + i * bytes, bytes, cudaMemcpyDeviceToHost, si)) != cudaSuccess)
        return e;
      if ((e = cudaEventRecord(P->out_ev[i + 1], si)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s, P->out_ev[i + 1], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // The host-buffer cycle with the copy in overlapped too (one group, FP32
  // paired kernel, no learned step, refinement source or smoother): psi
  // arrives in kOutParts direction ranges on the side streams, and each
  // range's scalar-flux partials and its residual with zero source (-A psi)
  // run as soon as it is in; then the source b, the restriction to level 1
  // that forms r = b - A psi on the way (bit for bit the residual kernel's
  // r, written back for the finest sweeps) with the residual norm, and the
  // rest of the cycle with the copy back of mg_cycle_host.  Returns
  // kNotPipelined, having queued nothing, when the problem does not qualify.
  static constexpr int kNotPipelined = 1;  // not a status (statuses are 0 or negative)
  static int mg_cycle_host_pipelined(btmg_problem* P, const void* h_in, void* h_out, double* rel, cudaStream_t s) {
    if constexpr (!(std::is_same<T, float>::value && std::is_same<C, float>::value)) {
      return kNotPipelined;
    } else {
      const LevelH &L0 = P->lev[0], &L1 = P->lev[P->L > 1 ? 1 : 0];
      if (P->G != 1 || P->d.pg == 0 || P->learned || P->inner_extra || P->zero_src || P->d.scat_levels != 0 ||
          P->L < 2 || P->plain_tail < 1 || P->nchunk % kOutParts != 0)
        return kNotPipelined;
      PgArgs<T, C> a = pg_args(P, 0, dptr<T>(P->d_hpsi));
      a.b = dptr<C>(P->d_hzero);
      a.extra = nullptr;
      a.r_out = dptr<C>(P->d_s[0]);
      a.norm_part = P->d_norm_part;  // the range launches' partials are not used
      int nparts = 0;
      if (!pg2_applies(a) || !restrict_rb_applies(L0.nx, L0.ny, L0.nr, L0.nc, L1.nx, L1.ny, L1.nr, L1.nc, L0.fx,
                                                  L0.fy, L0.fr, L0.fc, 1 << 24, &nparts))
        return kNotPipelined;
      if (!P->d_hparts) {
        CK(cudaMalloc(&P->d_hparts, (size_t)nparts * sizeof(double)));
        P->n_hparts = nparts;
      }
      const size_t plane = L0.npix() * sizeof(T);
      const int per = P->nchunk / kOutParts;
      const size_t rbytes = (size_t)per * P->dpc * plane;
      CK(cudaEventRecord(P->out_ev[0], s));
      for (int i = 0; i < kOutParts; ++i) {
        cudaStream_t si = P->out_s[i];
        const size_t n0 = (size_t)i * per * P->dpc;  // first direction of the range
        CK(cudaStreamWaitEvent(si, P->out_ev[0], 0));
        CK(cudaMemcpyAsync(reinterpret_cast<char*>(P->d_hpsi) + i * rbytes,
                           reinterpret_cast<const char*>(h_in) + i * rbytes, rbytes, cudaMemcpyHostToDevice, si));
        CK(launch_phi_partial<T, C>(dptr<T>(P->d_hpsi) + n0 * L0.npix(),
                                    dptr<C>(P->d_phi_part) + (size_t)i * per * L0.npix(),
                                    reinterpret_cast<const Dir<C>*>(P->d_dir[0]) + n0, L0.nx, L0.ny,
                                    per * P->dpc, P->dpc, per, si));
        PgArgs<T, C> ai = a;
        ai.chunk0 = i * per;
        CK(launch_pg<T, C>(ai, PG_RESID, true, per, si));
        CK(cudaEventRecord(P->out_ev[i + 1], si));
        CK(cudaStreamWaitEvent(s, P->out_ev[i + 1], 0));
      }
      CK(source(P, 0, s, true, false));
      CK(launch_restrict_rb(dptr<C>(P->d_s[0]), dptr<C>(P->d_b), dptr<C>(P->d_s[1]), dptr<C>(P->d_rcoef[0]),
                            reinterpret_cast<const Dir<C>*>(P->d_dir[0]), L0.dx * L0.dy, P->d_hparts, L0.nx,
                            L0.ny, L0.nr, L0.nc, L1.nx, L1.ny, L1.nr, L1.nc, s));
      CK(launch_sum2(P->d_hparts, P->n_hparts, P->d_rn2, P->d_qn2_part, P->n_q_blocks, P->d_qn2, s));
      P->out_host = h_out;
      P->first_restricted = true;
      const cudaError_t e = cycle_part_b(P, dptr<T>(P->d_hpsi), 0, s);
      P->first_restricted = false;
      P->out_host = nullptr;
      CK(e);
      return rel ? read_rel(P, s, 0, nullptr, rel) : BTMG_OK;
    }
  }

  // One cycle on host buffers: psi_in to the device copy, the cycle, every
  // group's result streamed to psi_out as its final launch completes (a
  // cycle with the learned step changes psi after that launch: its copy
  // follows the whole cycle instead).
  static int mg_cycle_host(btmg_problem* P, const void* h_in, void* h_out, double* rel, cudaStream_t s) {
    const size_t bytes = (size_t)P->G * P->lev[0].n() * sizeof(T);
    if (!P->d_hpsi) CK(cudaMalloc(&P->d_hpsi, bytes));
    for (int i = 0; i < kOutParts; ++i)
      if (!P->out_s[i]) CK(cudaStreamCreateWithFlags(&P->out_s[i], cudaStreamNonBlocking));
    for (int i = 0; i <= kOutParts; ++i)
      if (!P->out_ev[i]) CK(cudaEventCreateWithFlags(&P->out_ev[i], cudaEventDisableTiming));
    if (!P->d_hzero) {
      CK(cudaMalloc(&P->d_hzero, P->lev[0].npix() * sizeof(C)));
      CK(cudaMemsetAsync(P->d_hzero, 0, P->lev[0].npix() * sizeof(C), s));
    }
    const int prc = mg_cycle_host_pipelined(P, h_in, h_out, rel, s);
    if (prc != kNotPipelined) return prc;
    CK(cudaMemcpyAsync(P->d_hpsi, h_in, bytes, cudaMemcpyHostToDevice, s));
    if (P->learned) {
      if (int rc = mg_cycle(P, P->d_hpsi, nullptr, s)) return rc;
      CK(cudaMemcpyAsync(h_out, P->d_hpsi, bytes, cudaMemcpyDeviceToHost, s));
      return rel ? read_rel(P, s, 0, nullptr, rel) : BTMG_OK;
    }
    P->out_host = h_out;
    const int rc = mg_cycle(P, P->d_hpsi, rel, s);
    P->out_host = nullptr;
    return rc;
  }

  static int cycle_group(btmg_problem* P, T* psi_g, int g, cudaStream_t s, bool learn = false) {
    if (learn) return cycle_learned(P, psi_g, g, s);
    CK(cycle_part_a(P, psi_g, g, s));
    CK(cycle_part_b(P, psi_g, g, s));
    return BTMG_OK;
  }

  // residual of the correction in d_lc (zero external source) into r_out;
  // with `norm_to`, its weighted squared norm there
  static int homog_residual(btmg_problem* P, int g, C* r_out, double* norm_to, cudaStream_t s) {
    PgArgs<T, C> a = pg_args(P, g, dptr<T>(P->d_lc));
    a.b = dptr<C>(P->d_lb);
    a.extra = nullptr;
    a.r_out = r_out;
    a.norm_part = P->d_norm_part;
    CK(timed(P, PC_PG_RESID, s, [&] { return launch_pg<T, C>(a, PG_RESID, P->d.pg != 0, P->nchunk, s); }));
    if (norm_to) {
      CK(timed(P, PC_MISC, s, [&] { return launch_sum(P->d_norm_part, P->n_norm_sum, norm_to, s); }));
    }
    return BTMG_OK;
  }

  // A cycle of group g with the learned step (plain multigrid stays the
  // arbiter and the fallback):
  //  1. phi0 = scalar flux of psi; psi' = the plain cycle of psi;
  //  2. r' = residual of psi', rho' = sum_n p_n r'_n;
  //  3. the U-net predicts the shape of the scalar-flux error e of psi' from
  //     rho', the materials and the cycle's update phi(psi') - phi0, all
  //     averaged over lf x lf nodes (a canvas of at most 64 x 64 pixels, so
  //     the net sees the whole domain and its cost does not grow with the
  //     grid); c = the P1 angular flux of e interpolated to the fine nodes,
  //     b_c its scattering source;
  //  4. c' = M c, the plain cycle applied to c with zero source (M = the
  //     cycle's error propagation, which damps the small-scale part of the
  //     prediction as it damps the error of psi);
  //  5. rc = residual of c' (= -L c');
  //  6. psi' += alpha c' with alpha = -<r', rc>_W / <rc, rc>_W, which
  //     minimises the weighted residual norm of psi' + alpha c' (alpha = 0,
  //     the plain cycle, when the predicted gain is rounding noise; |alpha|
  //     capped so that the step's scalar flux stays within 1e3 times the
  //     cycle's own update).
  // Everything runs on the device, so the cycle can be graph-captured.  With
  // the nonlinear PG operator, step 6 uses the linearisation; the next cycle
  // evaluates the true residual.
  static int cycle_learned(btmg_problem* P, T* psi_g, int g, cudaStream_t s) {
    const LevelH& L0 = P->lev[0];
    const size_t npix = L0.npix();
    const C* sigt = dptr<C>(P->d_sig[0]) + (size_t)g * npix;
    const C* sigs = dptr<C>(P->d_sigs) + ((size_t)g * P->G + g) * npix;
    const Dir<C>* dir = reinterpret_cast<const Dir<C>*>(P->d_dir[0]);
    C* phi_g = dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * npix;
    CK(timed(P, PC_MISC, s, [&] { return launch_phi_sum<C>(phi_g, P->nchunk, (int)npix, dptr<C>(P->d_lphi0), s); }));
    CK(cycle_part_a(P, psi_g, g, s));
    CK(cycle_part_b(P, psi_g, g, s));
    CK(cycle_part_a(P, psi_g, g, s));
    CK(timed(P, PC_MISC, s, [&] {
      return launch_learn_features<C>(dptr<C>(P->d_rho_part) + (size_t)g * P->nchunk * npix, P->nchunk, phi_g,
                                      dptr<C>(P->d_lphi0), sigt, sigs, L0.dx, L0.nx, L0.ny, P->lf, P->W8, P->H8,
                                      P->d_lsum, P->d_lpart, P->d_feat, P->d_lscale, s);
    }));
    CK(timed(P, PC_MISC, s, [&] {
      return launch_dphi_norm<C>(phi_g, P->nchunk, dptr<C>(P->d_lphi0), (int)npix, P->d_ldpart, kDotBlocks,
                                 P->d_ldot + 3, s);
    }));
    if (int rc = btmg_unet_forward(P->learned, P->d_feat, P->d_dimg, 1, P->H8, P->W8, s))
      return fail(rc, std::string("learned correction: ") + btmg_unet_last_error());
    const double len = std::max(P->d.lx, P->d.ly);
    CK(timed(P, PC_MISC, s, [&] {
      return launch_learn_build<T, C>(dptr<T>(P->d_lc), dptr<C>(P->d_lb), P->d_dimg, sigt, sigs, dir, L0.nd, L0.nx,
                                      L0.ny, P->lf, P->W8, L0.dx, L0.dy, len > 0 ? 1.0 / len : 0.0, s);
    }));
    // r' stays in d_lr while the cycle of c uses the level-0 residual buffer
    CK(cudaMemcpyAsync(P->d_lr, P->d_s[0], L0.n() * sizeof(C), cudaMemcpyDeviceToDevice, s));
    if (int rc = homog_residual(P, g, dptr<C>(P->d_s[0]), nullptr, s)) return rc;
    CK(cycle_part_b(P, dptr<T>(P->d_lc), g, s, true));
    CK(homog_source(P, g, s));
    if (int rc = homog_residual(P, g, dptr<C>(P->d_s[0]), P->d_ldot + 1, s)) return rc;
    CK(timed(P, PC_MISC, s, [&] {
      return launch_dphi_norm<C>(dptr<C>(P->d_lphi), P->nchunk, dptr<C>(P->d_lzero), (int)npix, P->d_ldpart,
                                 kDotBlocks, P->d_ldot + 2, s);
    }));
    CK(timed(P, PC_MISC, s, [&] {
      return launch_learn_dot<C>(dptr<C>(P->d_lr), dptr<C>(P->d_s[0]), dir, L0.nx, L0.ny, L0.nd, L0.dx * L0.dy,
                                 P->d_ldpart, kDotBlocks, P->d_ldot, s);
    }));
    CK(timed(P, PC_MISC, s, [&] {
      return launch_learn_update<T, C>(psi_g, dptr<T>(P->d_lc), L0.n(), phi_g, dptr<C>(P->d_lphi),
                                       (size_t)P->nchunk * npix, P->d_ldot, P->d_rn2 + g, P->d_lstat, s);
    }));
    return BTMG_OK;
  }

  static int mg_cycle(btmg_problem* P, void* psi, double* rel, cudaStream_t s) {
    T* ps = reinterpret_cast<T*>(psi);
    CK(phi_partials(P, ps, s));
    const bool learn = P->learned && !P->learn_off && (P->learn_count++ % P->learn_every) == 0;
    for (int g = 0; g < P->G; ++g) {
      if (int rc = cycle_group(P, ps + (size_t)g * P->lev[0].n(), g, s, learn)) return rc;
    }
    if (rel) {
      CK(cudaMemcpyAsync(P->h_pinned, P->d_rn2, sizeof(double) * P->G, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(P->h_pinned + P->G, P->d_qn2, sizeof(double) * P->G, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(P->h_pinned + 2 * P->G, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*reinterpret_cast<int*>(P->h_pinned + 2 * P->G)) return fail(BTMG_ERR_TIMEOUT, "a bounded device wait gave up");
      double sr = 0, sq = 0;
      for (int g = 0; g < P->G; ++g) {
        sr += P->h_pinned[g];
        sq += P->h_pinned[P->G + g];
      }
      *rel = sq > 0 ? std::sqrt(sr / (4.0 * kPi * P->lev[0].dx * P->lev[0].dy * sq)) : std::sqrt(sr);
    }
    return BTMG_OK;
  }

  // residual of every group of psi; norms into d_rn2/d_qn2, r to r_out if non-null
  static cudaError_t residual_all(btmg_problem* P, const T* psi, C* r_out, cudaStream_t s) {
    cudaError_t e;
    if ((e = phi_partials(P, psi, s)) != cudaSuccess) return e;
    const LevelH& L0 = P->lev[0];
    for (int g = 0; g < P->G; ++g) {
      if ((e = source(P, g, s)) != cudaSuccess) return e;
      PgArgs<T, C> a = pg_args(P, g, psi + (size_t)g * L0.n());
      a.r_out = r_out ? r_out + (size_t)g * L0.n() : dptr<C>(P->d_s[0]);
      a.norm_part = P->d_norm_part;
      if ((e = launch_pg<T, C>(a, PG_RESID, P->d.pg != 0, P->nchunk, s)) != cudaSuccess) return e;
      if ((e = launch_sum(P->d_norm_part, P->n_norm_sum, P->d_rn2 + g, s)) != cudaSuccess)
        return e;
    }
    return cudaSuccess;
  }

  static int read_rel(btmg_problem* P, cudaStream_t s, int g, double* rel_g, double* rel_all) {
    CK(cudaMemcpyAsync(P->h_pinned, P->d_rn2, sizeof(double) * P->G, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(P->h_pinned + P->G, P->d_qn2, sizeof(double) * P->G, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(P->h_pinned + 2 * P->G, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*reinterpret_cast<int*>(P->h_pinned + 2 * P->G)) return fail(BTMG_ERR_TIMEOUT, "a bounded device wait gave up");
    const double w = 4.0 * kPi * P->lev[0].dx * P->lev[0].dy;
    if (rel_g) {
      const double rn = P->h_pinned[g], qn = P->h_pinned[P->G + g];
      *rel_g = qn > 0 ? std::sqrt(rn / (w * qn)) : std::sqrt(rn);
    }
    if (rel_all) {
      double sr = 0, sq = 0;
      for (int h = 0; h < P->G; ++h) {
        sr += P->h_pinned[h];
        sq += P->h_pinned[P->G + h];
      }
      *rel_all = sq > 0 ? std::sqrt(sr / (w * sq)) : std::sqrt(sr);
    }
    return BTMG_OK;
  }

  static int solve(btmg_problem* P, void* psi, double rtol, int max_cycles, btmg_solve_info* info, cudaStream_t s) {
    if (!s) {
      CK(cudaEventRecord(P->order_event, s));
      CK(cudaStreamWaitEvent(P->own_stream, P->order_event, 0));
      s = P->own_stream;
    }
    T* ps = reinterpret_cast<T*>(psi);
    const int check = (info && info->check_every > 0) ? info->check_every : 1;
    if (P->graph_psi != psi || P->graph_stream != s) free_graphs(P);
    P->learn_off = false;
    P->scat_off = false;
    int cycles = 0, status = BTMG_OK;
    CK(phi_partials(P, ps, s));
    int max_outer = (info && info->max_outer > 0) ? info->max_outer : (P->upscatter ? 8 : 1);
    if (P->G == 1) max_outer = 1;
    double rel_all = 0.0;
    for (int outer = 0; outer < max_outer; ++outer) {
      for (int g = 0; g < P->G; ++g) {
        T* pg = ps + (size_t)g * P->lev[0].n();
        double best = 1e300;
        bool warm[2] = {false, false};
        for (int c = 0; c < max_cycles; ++c) {
          // the learned step runs in every learn_every-th cycle (from the first)
          const bool learn = P->learned && !P->learn_off && (c % P->learn_every) == 0;
          cudaGraphExec_t& ge = learn ? P->lgraphs[g] : P->graphs[g];
          if (!ge) {
            if (!warm[learn]) {
              // eager first cycle of each kind (sets kernel attributes, sizes workspaces)
              warm[learn] = true;
              if (int rc = cycle_group(P, pg, g, s, learn)) return rc;
            } else {
              cudaGraph_t graph;
              CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
              int rc = cycle_group(P, pg, g, s, learn);
              cudaError_t ee = cudaStreamEndCapture(s, &graph);
              if (rc) return rc;
              CK(ee);
              cudaError_t ei = cudaGraphInstantiate(&ge, graph, 0);
              cudaGraphDestroy(graph);
              CK(ei);
              P->graph_psi = psi;
              P->graph_stream = s;
              CK(cudaGraphLaunch(ge, s));
            }
          } else {
            CK(cudaGraphLaunch(ge, s));
          }
          ++cycles;
          if ((c + 1) % check == 0 || c + 1 == max_cycles) {
            double rel;
            int rc = read_rel(P, s, g, &rel, nullptr);
            if (rc) return rc;
            if (info && info->history && cycles - 1 < info->history_len) info->history[cycles - 1] = rel;
            if (std::isnan(rel)) {
              status = BTMG_ERR_NAN;
              break;
            }
            if (rel > 1e3 * best && best < 1e299) {
              status = BTMG_ERR_DIVERGED;
              break;
            }
            // plain multigrid is the arbiter of the learned step: a residual above
            // twice the best so far ends it for the rest of this solve
            if (P->learned && !P->learn_off && best < 1e299 && rel > 2.0 * best) {
              P->learn_off = true;
              ++P->learn_fallbacks;
            }
            // and the scattering smoother likewise: the rest of this solve
            // runs the published cycle (recaptured, first cycle eager)
            if (P->d.scat_levels && !P->scat_off && best < 1e299 && rel > 2.0 * best) {
              P->scat_off = true;
              ++P->scat_fallbacks;
              free_graphs(P);
              warm[0] = warm[1] = false;
            }
            if (rel < best) best = rel;
            if (rel <= rtol) break;
          }
        }
        if (status != BTMG_OK) break;
      }
      if (status != BTMG_OK) break;
      CK(residual_all(P, ps, nullptr, s));
      int rc = read_rel(P, s, 0, nullptr, &rel_all);
      if (rc) return rc;
      if (rel_all <= rtol || outer + 1 == max_outer) break;
      CK(phi_partials(P, ps, s));
    }
    if (status == BTMG_OK && !(rel_all <= rtol)) status = std::isnan(rel_all) ? BTMG_ERR_NAN : BTMG_ERR_NOT_CONVERGED;
    if (P->scat_off) {  // later calls start with the smoother again
      P->scat_off = false;
      free_graphs(P);
    }
    if (info) {
      info->cycles = cycles;
      info->rel_resid = rel_all;
      info->status = status;
    }
    return status;
  }
};

// Mixed-precision iterative refinement (linear fine operator, pg = 0):
//   r64 = b - A psi64 in FP64 (the FP64 twin's kernels);
//   solve A delta = alpha r64 approximately with `inner` low-precision
//   cycles from delta = 0 (psi stored in the problem's storage type, FP32
//   accumulation, external source 0, alpha = 1 / rms(r64) so the correction
//   is O(1) in BF16/FP16 range);  psi64 += delta / alpha.
template <typename T, typename C>
int refine_solve(btmg_problem* P, double* psi64, double rtol, int max_outer, int inner, btmg_solve_info* info,
                 cudaStream_t s) {
  const LevelH& L0 = P->lev[0];
  const size_t n_all = (size_t)P->G * L0.n(), npix = L0.npix();
  if (!P->twin) {
    btmg_problem_desc d2 = P->d;
    d2.region = P->h_region.data();
    d2.sigma_t = P->h_sigma_t.data();
    d2.sigma_s = P->h_sigma_s.data();
    d2.source = P->h_source.data();
    d2.psi_dtype = BTMG_F64;
    d2.max_levels = 1;
    d2.scat_levels = 0;  // residuals only
    int rc = create(&d2, &P->twin);
    if (rc) return rc;
  }
  if (!P->d_delta_all) {
    CK(cudaMalloc(&P->d_delta_all, n_all * sizeof(T)));
    CK(cudaMalloc(&P->d_extra_all, n_all * sizeof(C)));
    CK(cudaMalloc(&P->d_r64, n_all * sizeof(double)));
    CK(cudaMalloc(&P->d_zero_src, (size_t)P->G * npix * sizeof(C)));
    CK(cudaMemsetAsync(P->d_zero_src, 0, (size_t)P->G * npix * sizeof(C), s));
  }
  btmg_problem* Q = P->twin;
  const double w = 4.0 * kPi * L0.dx * L0.dy;
  int cycles = 0, status = BTMG_ERR_NOT_CONVERGED;
  double rel = 0.0, best = 1e300;
  P->learn_off = false;
  P->scat_off = false;
  for (int outer = 0; outer <= max_outer; ++outer) {
    CK(Impl<double, double>::residual_all(Q, psi64, P->d_r64, s));
    int rc = Impl<double, double>::read_rel(Q, s, 0, nullptr, &rel);
    if (rc) return rc;
    if (info && info->history && outer < info->history_len) info->history[outer] = rel;
    if (std::isnan(rel)) {
      status = BTMG_ERR_NAN;
      break;
    }
    if (rel <= rtol) {
      status = BTMG_OK;
      break;
    }
    if (outer == max_outer) break;
    // plain multigrid is the arbiter of the learned step: an outer residual above 1.5
    // times the best so far ends it for the rest of this solve
    if (P->learned && !P->learn_off && rel > 1.5 * best) {
      P->learn_off = true;
      ++P->learn_fallbacks;
    }
    if (P->d.scat_levels && !P->scat_off && rel > 1.5 * best) {  // and the scattering smoother
      P->scat_off = true;
      ++P->scat_fallbacks;
      free_graphs(P);
    }
    if (rel < best) best = rel;
    double rn2 = 0.0;
    for (int g = 0; g < P->G; ++g) rn2 += Q->h_pinned[g];
    const double rms = std::sqrt(rn2 / (w * (double)npix * P->G));
    const double alpha = rms > 0 ? 1.0 / rms : 1.0;
    CK(launch_scale_to<C>(P->d_r64, dptr<C>(P->d_extra_all), alpha, n_all, s));
    CK(cudaMemsetAsync(P->d_delta_all, 0, n_all * sizeof(T), s));
    P->inner_extra = P->d_extra_all;
    P->zero_src = true;
    int rc2 = BTMG_OK;
    for (int k = 0; k < inner && rc2 == BTMG_OK; ++k) rc2 = Impl<T, C>::mg_cycle(P, P->d_delta_all, nullptr, s);
    P->inner_extra = nullptr;
    P->zero_src = false;
    if (rc2) return rc2;
    cycles += inner;
    CK(launch_refine_update<T>(psi64, dptr<T>(P->d_delta_all), 1.0 / alpha, n_all, s));
  }
  CK(cudaStreamSynchronize(s));
  if (P->scat_off) {  // later calls start with the smoother again
    P->scat_off = false;
    free_graphs(P);
  }
  if (info) {
    info->cycles = cycles;
    info->rel_resid = rel;
    info->status = status;
  }
  return status;
}

// features of the learned step for psi (training pairs), per group
template <typename T, typename C> struct RunFeatures {
  static int run(btmg_problem* P, const void* psi, const void* psi_prev, float* feat, float* scale, cudaStream_t s) {
    const T* ps = reinterpret_cast<const T*>(psi);
    const LevelH& L0 = P->lev[0];
    const size_t npix = L0.npix();
    const size_t nf = (size_t)P->H8 * P->W8 * kLearnFeatures;
    if (psi_prev) {  // scalar flux of psi_prev per group into the (G-sized) zero-source scratch
      CK(Impl<T, C>::phi_partials(P, reinterpret_cast<const T*>(psi_prev), s));
      for (int g = 0; g < P->G; ++g)
        CK(launch_phi_sum<C>(dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * npix, P->nchunk, (int)npix,
                             dptr<C>(P->d_lprev_all) + (size_t)g * npix, s));
    }
    CK(Impl<T, C>::phi_partials(P, ps, s));
    for (int g = 0; g < P->G; ++g) {
      CK(Impl<T, C>::source(P, g, s));
      PgArgs<T, C> a = Impl<T, C>::pg_args(P, g, ps + (size_t)g * L0.n());
      a.r_out = dptr<C>(P->d_s[0]);
      a.norm_part = P->d_norm_part;
      a.rho_part = dptr<C>(P->d_rho_part) + (size_t)g * P->nchunk * npix;
      CK(launch_pg<T, C>(a, PG_RESID, P->d.pg != 0, P->nchunk, s));
      CK(launch_learn_features<C>(a.rho_part, P->nchunk, dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * npix,
                                  psi_prev ? dptr<C>(P->d_lprev_all) + (size_t)g * npix : nullptr,
                                  dptr<C>(P->d_sig[0]) + (size_t)g * npix,
                                  dptr<C>(P->d_sigs) + ((size_t)g * P->G + g) * npix, L0.dx, L0.nx, L0.ny, P->lf,
                                  P->W8, P->H8, P->d_lsum, P->d_lpart, feat + (size_t)g * nf, scale + g, s));
    }
    return BTMG_OK;
  }
};

template <typename T, typename C> struct RunRefine {
  static int run(btmg_problem* P, double* psi64, double rtol, int mo, int inner, btmg_solve_info* info,
                 cudaStream_t s) {
    return refine_solve<T, C>(P, psi64, rtol, mo, inner, info, s);
  }
};

template <template <typename, typename> class F, typename... Args>
int dispatch(int dtype, Args&&... args) {
  switch (dtype) {
    case BTMG_F64: return F<double, double>::run(args...);
    case BTMG_F32: return F<float, float>::run(args...);
    case BTMG_BF16: return F<__nv_bfloat16, float>::run(args...);
    case BTMG_F16: return F<__half, float>::run(args...);
  }
  return fail(BTMG_ERR_INVALID_ARG, "unknown dtype");
}

template <typename T, typename C> struct RunCycle {
  static int run(btmg_problem* P, void* psi, double* rel, cudaStream_t s) { return Impl<T, C>::mg_cycle(P, psi, rel, s); }
};
template <typename T, typename C> struct RunCycleHost {
  static int run(btmg_problem* P, const void* in, void* out, double* rel, cudaStream_t s) {
    return Impl<T, C>::mg_cycle_host(P, in, out, rel, s);
  }
};
template <typename T, typename C> struct RunSolve {
  static int run(btmg_problem* P, void* psi, double rtol, int mc, btmg_solve_info* info, cudaStream_t s) {
    return Impl<T, C>::solve(P, psi, rtol, mc, info, s);
  }
};
template <typename T, typename C> struct RunApply {
  static int run(btmg_problem* P, const void* psi, void* r, cudaStream_t s) {
    CK(Impl<T, C>::residual_all(P, reinterpret_cast<const T*>(psi), reinterpret_cast<C*>(r), s));
    return BTMG_OK;
  }
};
template <typename T, typename C> struct RunFlux {
  static int run(btmg_problem* P, const void* psi, void* phi, cudaStream_t s) {
    CK(Impl<T, C>::phi_partials(P, reinterpret_cast<const T*>(psi), s));
    const size_t npix = P->lev[0].npix();
    for (int g = 0; g < P->G; ++g)
      CK(launch_phi_sum<C>(dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * npix, P->nchunk, (int)npix,
                           reinterpret_cast<C*>(phi) + g * npix, s));
    return BTMG_OK;
  }
};
template <typename T, typename C> struct RunSmoothPG {
  static int run(btmg_problem* P, void* psi, int sweeps, cudaStream_t s) {
    T* ps = reinterpret_cast<T*>(psi);
    const LevelH& L0 = P->lev[0];
    CK(Impl<T, C>::phi_partials(P, ps, s));
    for (int k = 0; k < sweeps; ++k)
      for (int g = 0; g < P->G; ++g) {
        CK(Impl<T, C>::source(P, g, s, false));
        PgArgs<T, C> j = Impl<T, C>::pg_args(P, g, ps + (size_t)g * L0.n());
        j.psi_out = dptr<T>(P->d_psi_tmp);
        j.phi_part = dptr<C>(P->d_phi_part) + (size_t)g * P->nchunk * L0.npix();
        CK(launch_pg<T, C>(j, PG_JACOBI, P->d.pg != 0, P->nchunk, s));
        CK(cudaMemcpyAsync(ps + (size_t)g * L0.n(), P->d_psi_tmp, L0.n() * sizeof(T), cudaMemcpyDeviceToDevice, s));
      }
    return BTMG_OK;
  }
};
template <typename T, typename C> struct RunSmoothUp {
  static int run(btmg_problem* P, void* psi, const void* src, int l, int g, int sweeps, cudaStream_t s) {
    const LevelH& A = P->lev[l];
    if (!P->d_delta[l]) CK(cudaMalloc(&P->d_delta[l], A.n() * sizeof(C)));
    if (P->scat_on[l] && sweeps > 0) {  // scattering smoother on this level
      CK(Impl<T, C>::scat_level(P, l, g, reinterpret_cast<const C*>(src), INIT_SAME, reinterpret_cast<const C*>(psi),
                                sweeps, nullptr, nullptr, nullptr, PC_UP_COARSE, s));
      CK(cudaMemcpyAsync(psi, P->d_delta[l], A.n() * sizeof(C), cudaMemcpyDeviceToDevice, s));
      return BTMG_OK;
    }
    int left = sweeps;
    while (left > 0) {
      const int k = left > 8 ? 8 : left;
      UpArgs<T, C> u = Impl<T, C>::up_args(P, l, g);
      u.nu = k;
      u.src = reinterpret_cast<const C*>(src);
      u.init_mode = INIT_SAME;
      u.init = reinterpret_cast<const C*>(psi);
      u.delta_out = dptr<C>(P->d_delta[l]);
      CK(launch_upwind<T, C>(u, UP_CORR, A.nd, s));
      CK(cudaMemcpyAsync(psi, P->d_delta[l], A.n() * sizeof(C), cudaMemcpyDeviceToDevice, s));
      left -= k;
    }
    return BTMG_OK;
  }
};

void destroy(btmg_problem* P) {
  if (!P) return;
  free_graphs(P);
  if (P->twin) destroy(P->twin);
  for (void* p : {P->d_zero_src, P->d_delta_all, P->d_extra_all, (void*)P->d_r64, P->d_rho_part, (void*)P->d_feat,
                  (void*)P->d_dimg, (void*)P->d_lscale, (void*)P->d_lsum, (void*)P->d_lpart, P->d_lc, P->d_lr, P->d_lb,
                  (void*)P->d_ldot, (void*)P->d_ldpart, (void*)P->d_lstat, P->d_lphi, P->d_lzero, P->d_lphi0,
                  P->d_lprev_all})
    if (p) cudaFree(p);
  for (cudaEvent_t e : P->prof_pool) cudaEventDestroy(e);
  for (auto v : {&P->d_dir, &P->d_rcoef, &P->d_sig, &P->d_s, &P->d_delta, &P->d_parent, &P->d_scat_w})
    for (void* p : *v)
      if (p) cudaFree(p);
  for (void* p : {P->d_scat_j, P->d_scat_part, P->d_scat_c, P->d_pgd})
    if (p) cudaFree(p);
  for (void* p : {P->d_sigs, P->d_src, P->d_b, P->d_phi_part, P->d_psi_tmp, (void*)P->d_norm_part, (void*)P->d_err,
                  (void*)P->d_qn2_part, (void*)P->d_rn2, (void*)P->d_qn2})
    if (p) cudaFree(p);
  if (P->h_pinned) cudaFreeHost(P->h_pinned);
  if (P->own_stream) cudaStreamDestroy(P->own_stream);
  for (auto& st : P->out_s)
    if (st) cudaStreamDestroy(st);
  for (auto& ev : P->out_ev)
    if (ev) cudaEventDestroy(ev);
  if (P->d_hpsi) cudaFree(P->d_hpsi);
  if (P->d_hzero) cudaFree(P->d_hzero);
  if (P->d_hparts) cudaFree(P->d_hparts);
  if (P->order_event) cudaEventDestroy(P->order_event);
  delete P;
}

template <typename C> void put_dirs(std::vector<char>& buf, const LevelH& A) {
  buf.resize(sizeof(Dir<C>) * A.nd);
  Dir<C>* d = reinterpret_cast<Dir<C>*>(buf.data());
  for (int n = 0; n < A.nd; ++n) {
    d[n].mu = (C)A.mu[n];
    d[n].nu = (C)A.nu[n];
    d[n].w = (C)A.p[n];
    d[n].ax = (C)(std::fabs(A.mu[n]) / A.dx);
    d[n].ay = (C)(std::fabs(A.nu[n]) / A.dy);
  }
}

template <typename C> void put_vals(std::vector<char>& buf, const std::vector<double>& v) {
  buf.resize(sizeof(C) * v.size());
  C* d = reinterpret_cast<C*>(buf.data());
  for (size_t i = 0; i < v.size(); ++i) d[i] = (C)v[i];
}

int upload(void** dst, const std::vector<char>& buf) {
  CK(cudaMalloc(dst, buf.size() ? buf.size() : 8));
  if (buf.size()) CK(cudaMemcpy(*dst, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  return BTMG_OK;
}

// Direction chunks: the PG grid is tiles x chunks CTAs; pick the divisor of nd
// (at most 64 chunks) whose grid comes closest to whole waves of resident
// CTAs, preferring fewer chunks on ties (fewer flux partials).
int auto_chunks(int dtype, bool pg, int tiles, int nd) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int occ = 1;
  switch (dtype) {
    case BTMG_F64: occ = pg_blocks_per_sm<double, double>(pg); break;
    case BTMG_F32: occ = pg_blocks_per_sm<float, float>(pg); break;
    case BTMG_BF16: occ = pg_blocks_per_sm<__nv_bfloat16, float>(pg); break;
    default: occ = pg_blocks_per_sm<__half, float>(pg); break;
  }
  const double slots = (double)sms * occ;
  int best = 1;
  double best_eff = -1.0;
  for (int c = 1; c <= nd && c <= 64; ++c) {
    if (nd % c) continue;
    if (dtype == BTMG_F32 && pg && (nd / c) % 2) continue;  // the FP32 PG kernel takes direction pairs
    const double items = (double)tiles * c;
    const double waves = std::ceil(items / slots);
    const double eff = items / (waves * slots);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = c;
    }
  }
  return best;
}

int create(const btmg_problem_desc* d, btmg_problem** out) {
  if (!d || !out) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nx > 65536 || d->ny > 65536 || !(d->lx > 0) || !(d->ly > 0))
    return fail(BTMG_ERR_INVALID_ARG, "bad grid size");
  if (d->n_polar < 2 || d->n_polar % 2 || d->n_azim < 4 || d->n_azim % 4)
    return fail(BTMG_ERR_INVALID_ARG, "n_polar must be even and n_azim a multiple of 4");
  if (d->n_groups < 1 || d->n_regions < 1 || !d->region || !d->sigma_t || !d->sigma_s || !d->source)
    return fail(BTMG_ERR_INVALID_ARG, "bad material description");
  if (d->psi_dtype < BTMG_F64 || d->psi_dtype > BTMG_F16) return fail(BTMG_ERR_INVALID_ARG, "bad psi_dtype");
  if (d->nu_jacobi < 1 || d->nu_jacobi > 8) return fail(BTMG_ERR_INVALID_ARG, "nu_jacobi must be in 1..8");
  {
    const int nd = d->n_polar * d->n_azim;  // 8 faces of (n_polar / 2) x (n_azim / 4)
    if (d->chunks < 0 || d->chunks > 64 || (d->chunks > 0 && nd % d->chunks))
      return fail(BTMG_ERR_INVALID_ARG, "chunks must be 0 or a divisor of the direction count, at most 64");
  }
  if (d->order < 1 || d->order > 3) return fail(BTMG_ERR_INVALID_ARG, "order must be 1, 2 or 3");
  if (d->pg && d->order == 1 && d->psi_dtype > BTMG_F32)
    return fail(BTMG_ERR_UNSUPPORTED, "the linear-order PG operator is built for FP64 and FP32 storage");
  for (int i = 0; i < 4; ++i)
    if (d->bc[i] != BTMG_VACUUM && d->bc[i] != BTMG_REFLECTIVE) return fail(BTMG_ERR_INVALID_ARG, "bad bc");
  const int G = d->n_groups, nx = d->nx, ny = d->ny;
  const size_t npix = (size_t)nx * ny;
  for (size_t i = 0; i < npix; ++i)
    if (d->region[i] < 0 || d->region[i] >= d->n_regions) return fail(BTMG_ERR_INVALID_ARG, "region id out of range");
  // materials: finite, cross sections non-negative (sigma_t = 0 is a void)
  for (size_t i = 0; i < (size_t)d->n_regions * G; ++i) {
    if (!std::isfinite(d->sigma_t[i]) || d->sigma_t[i] < 0.0 || !std::isfinite(d->source[i]))
      return fail(BTMG_ERR_INVALID_ARG, "sigma_t must be finite and >= 0, the source finite");
  }
  for (size_t i = 0; i < (size_t)d->n_regions * G * G; ++i)
    if (!std::isfinite(d->sigma_s[i]) || d->sigma_s[i] < 0.0)
      return fail(BTMG_ERR_INVALID_ARG, "sigma_s must be finite and >= 0");
  if (d->scat_levels < 0 || d->scat_levels > 2) return fail(BTMG_ERR_INVALID_ARG, "scat_levels must be 0, 1 or 2");
  if (d->scat_levels)
    for (int r = 0; r < d->n_regions; ++r)
      for (int g = 0; g < G; ++g)
        if (d->sigma_s[((size_t)r * G + g) * G + g] > d->sigma_t[(size_t)r * G + g])
          return fail(BTMG_ERR_INVALID_ARG, "the scattering smoother needs sigma_s,gg <= sigma_t");

  btmg_problem* P = new btmg_problem();
  P->d = *d;
  P->h_region.assign(d->region, d->region + npix);
  P->h_sigma_t.assign(d->sigma_t, d->sigma_t + (size_t)d->n_regions * G);
  P->h_sigma_s.assign(d->sigma_s, d->sigma_s + (size_t)d->n_regions * G * G);
  P->h_source.assign(d->source, d->source + (size_t)d->n_regions * G);
  P->d.region = nullptr;
  P->d.sigma_t = P->d.sigma_s = P->d.source = nullptr;
  if (!(P->d.beta_pg > 0)) P->d.beta_pg = 3.0;
  P->G = G;
  P->dtype = d->psi_dtype;
  P->f64 = d->psi_dtype == BTMG_F64;
  P->csize = P->f64 ? 8 : 4;

  // finest level
  LevelH L0;
  L0.nx = nx;
  L0.ny = ny;
  L0.nr = d->n_polar / 2;
  L0.nc = d->n_azim / 4;
  L0.nd = 8 * L0.nr * L0.nc;
  L0.dx = d->lx / nx;
  L0.dy = d->ly / ny;
  octahedral_quadrature(L0.nr, L0.nc, L0.mu, L0.nu, L0.p);
  L0.sig.resize((size_t)G * npix);
  std::vector<double> sigs((size_t)G * G * npix), src((size_t)G * npix);
  for (size_t i = 0; i < npix; ++i) {
    const int rg = d->region[i];
    for (int g = 0; g < G; ++g) {
      L0.sig[(size_t)g * npix + i] = d->sigma_t[rg * G + g];
      src[(size_t)g * npix + i] = d->source[rg * G + g];
      for (int h = 0; h < G; ++h) sigs[((size_t)g * G + h) * npix + i] = d->sigma_s[((size_t)rg * G + g) * G + h];
    }
  }
  P->lev.push_back(L0);
  // coarser levels: each of nx, ny, nr, nc halves (ceil) until 1
  while (true) {
    LevelH& A = P->lev.back();
    if (d->max_levels > 0 && (int)P->lev.size() >= d->max_levels) break;
    if (A.nx == 1 && A.ny == 1 && A.nr == 1 && A.nc == 1) break;
    A.fx = A.nx > 1 ? 2 : 1;
    A.fy = A.ny > 1 ? 2 : 1;
    A.fr = A.nr > 1 ? 2 : 1;
    A.fc = A.nc > 1 ? 2 : 1;
    LevelH B;
    B.nx = (A.nx + A.fx - 1) / A.fx;
    B.ny = (A.ny + A.fy - 1) / A.fy;
    B.nr = (A.nr + A.fr - 1) / A.fr;
    B.nc = (A.nc + A.fc - 1) / A.fc;
    B.nd = 8 * B.nr * B.nc;
    B.dx = A.dx * A.fx;
    B.dy = A.dy * A.fy;
    B.mu.assign(B.nd, 0.0);
    B.nu.assign(B.nd, 0.0);
    B.p.assign(B.nd, 0.0);
    for (int n = 0; n < A.nd; ++n) {  // merged patches: summed weight, weighted mean direction
      const int f = n / (A.nr * A.nc), j = (n % (A.nr * A.nc)) / A.nc, i = n % A.nc;
      const int N = f * B.nr * B.nc + (j / A.fr) * B.nc + i / A.fc;
      B.p[N] += A.p[n];
      B.mu[N] += A.p[n] * A.mu[n];
      B.nu[N] += A.p[n] * A.nu[n];
    }
    for (int N = 0; N < B.nd; ++N) {
      B.mu[N] /= B.p[N];
      B.nu[N] /= B.p[N];
    }
    B.sig.assign((size_t)G * B.npix(), 0.0);
    for (int g = 0; g < G; ++g)
      for (int Y = 0; Y < B.ny; ++Y)
        for (int X = 0; X < B.nx; ++X) {  // harmonic mean of the present children, 0 if any is 0
          int cnt = 0;
          bool zero = false;
          double inv = 0.0;
          for (int yy = 0; yy < A.fy; ++yy)
            for (int xx = 0; xx < A.fx; ++xx) {
              const int x = X * A.fx + xx, y = Y * A.fy + yy;
              if (x >= A.nx || y >= A.ny) continue;
              const double v = A.sig[(size_t)g * A.npix() + (size_t)y * A.nx + x];
              ++cnt;
              if (v == 0.0) zero = true;
              else inv += 1.0 / v;
            }
          B.sig[(size_t)g * B.npix() + (size_t)Y * B.nx + X] = zero ? 0.0 : cnt / inv;
        }
    P->lev.push_back(B);
  }
  P->L = (int)P->lev.size();
  {  // the coarsest levels that fit the single-CTA tail kernel (not level 0)
    const size_t tmax = (size_t)(P->f64 ? scat_tail_max<double>() : scat_tail_max<float>());
    P->plain_tail = P->L;
    while (P->plain_tail - 1 >= 1 && P->L - (P->plain_tail - 1) <= kScatTailLevels &&
           P->lev[P->plain_tail - 1].n() <= tmax)
      --P->plain_tail;
  }
  for (int r = 0; r < d->n_regions; ++r)
    for (int g = 0; g < G; ++g)
      for (int h = g + 1; h < G; ++h)
        if (d->sigma_s[((size_t)r * G + g) * G + h] != 0.0) P->upscatter = true;
  // direction chunks of the fine level: enough CTAs to fill 152 SMs
  const LevelH& F = P->lev[0];
  P->tiles_x = (F.nx + kTile - 1) / kTile;
  P->tiles_y = (F.ny + kTile - 1) / kTile;
  const int tiles = P->tiles_x * P->tiles_y;
  {
    const int best = auto_chunks(P->dtype, d->pg != 0, tiles, F.nd);
    P->nchunk = d->chunks > 0 ? d->chunks : best;
    P->dpc = F.nd / P->nchunk;
  }
  P->graphs.assign(G, nullptr);

  int rc = BTMG_OK;
  auto bail = [&](int code) {
    destroy(P);
    return code;
  };
  std::vector<char> buf;
  P->d_dir.assign(P->L, nullptr);
  P->d_rcoef.assign(P->L, nullptr);
  P->d_sig.assign(P->L, nullptr);
  P->d_s.assign(P->L, nullptr);
  P->d_delta.assign(P->L, nullptr);
  P->d_parent.assign(P->L, nullptr);
  for (int l = 0; l < P->L; ++l) {
    const LevelH& A = P->lev[l];
    if (P->f64) put_dirs<double>(buf, A);
    else put_dirs<float>(buf, A);
    if ((rc = upload(&P->d_dir[l], buf))) return bail(rc);
    if (P->f64) put_vals<double>(buf, A.sig);
    else put_vals<float>(buf, A.sig);
    if ((rc = upload(&P->d_sig[l], buf))) return bail(rc);
    if (l + 1 < P->L) {  // restriction weights p_n dx dy / (P_N dX dY)
      const LevelH& B = P->lev[l + 1];
      std::vector<double> rc_(A.nd);
      for (int n = 0; n < A.nd; ++n) {
        const int f = n / (A.nr * A.nc), j = (n % (A.nr * A.nc)) / A.nc, i = n % A.nc;
        const int N = f * B.nr * B.nc + (j / A.fr) * B.nc + i / A.fc;
        rc_[n] = A.p[n] * A.dx * A.dy / (B.p[N] * B.dx * B.dy);
      }
      if (P->f64) put_vals<double>(buf, rc_);
      else put_vals<float>(buf, rc_);
      if ((rc = upload(&P->d_rcoef[l], buf))) return bail(rc);
      // parent (coarse) direction of every direction, for UpSamp
      buf.resize(sizeof(int) * A.nd);
      int* par = reinterpret_cast<int*>(buf.data());
      for (int n = 0; n < A.nd; ++n) {
        const int f = n / (A.nr * A.nc), j = (n % (A.nr * A.nc)) / A.nc, i = n % A.nc;
        par[n] = f * B.nr * B.nc + (j / A.fr) * B.nc + i / A.fc;
      }
      if ((rc = upload(&P->d_parent[l], buf))) return bail(rc);
    }
    if (cudaMalloc(&P->d_s[l], A.n() * P->csize) != cudaSuccess) return bail(fail(BTMG_ERR_OOM, "workspace s"));
    if (l >= 1 && cudaMalloc(&P->d_delta[l], A.n() * P->csize) != cudaSuccess)
      return bail(fail(BTMG_ERR_OOM, "workspace delta"));
  }
  // scattering smoother: the levels it runs on, the gain
  // w = kappa / (1 - kappa sum_n p_n / d_n) per level and group (kappa =
  // sigma_s / (4 pi), coarse sigma_s = harmonic sigma_t x the mean child
  // ratio sigma_s / sigma_t), sweep scratch for the largest smoothed level
  P->scat_on.assign(P->L, 0);
  P->d_scat_w.assign(P->L, nullptr);
  P->scat_tail = P->L;
  if (d->scat_levels) {
    std::vector<double> crat((size_t)G * npix, 0.0);
    for (size_t i = 0; i < npix; ++i)
      for (int g = 0; g < G; ++g) {
        const int rg = d->region[i];
        const double st = d->sigma_t[(size_t)rg * G + g];
        if (st > 0.0) crat[(size_t)g * npix + i] = d->sigma_s[((size_t)rg * G + g) * G + g] / st;
      }
    size_t max_n = 0, max_part = 0, max_pix = 0;
    for (int l = 0; l < P->L; ++l) {
      const LevelH& A = P->lev[l];
      if (l > 0) {  // mean over the present children
        const LevelH& F2 = P->lev[l - 1];
        std::vector<double> cc((size_t)G * A.npix(), 0.0);
        for (int g = 0; g < G; ++g)
          for (int Y = 0; Y < A.ny; ++Y)
            for (int X = 0; X < A.nx; ++X) {
              double acc = 0.0;
              int cnt = 0;
              for (int yy = 0; yy < F2.fy; ++yy)
                for (int xx = 0; xx < F2.fx; ++xx) {
                  const int x = X * F2.fx + xx, y = Y * F2.fy + yy;
                  if (x >= F2.nx || y >= F2.ny) continue;
                  acc += crat[(size_t)g * F2.npix() + (size_t)y * F2.nx + x];
                  ++cnt;
                }
              cc[(size_t)g * A.npix() + (size_t)Y * A.nx + X] = acc / cnt;
            }
        crat.swap(cc);
      }
      P->scat_on[l] = d->scat_levels == 2 || (A.nr == 1 && A.nc == 1);
      if (!P->scat_on[l]) continue;
      void* tmp = nullptr;
      if (P->f64) put_vals<double>(buf, crat);
      else put_vals<float>(buf, crat);
      if ((rc = upload(&tmp, buf))) return bail(rc);
      if (cudaMalloc(&P->d_scat_w[l], (size_t)G * A.npix() * P->csize) != cudaSuccess) {
        cudaFree(tmp);
        return bail(fail(BTMG_ERR_OOM, "scattering smoother gain"));
      }
      cudaError_t ge = cudaSuccess;
      for (int g = 0; g < G && ge == cudaSuccess; ++g) {
        const size_t o = (size_t)g * A.npix();
        ge = P->f64 ? launch_scat_gain<double>(dptr<double>(P->d_sig[l]) + o, dptr<double>(tmp) + o,
                                               reinterpret_cast<const Dir<double>*>(P->d_dir[l]), A.nd,
                                               (int)A.npix(), dptr<double>(P->d_scat_w[l]) + o, 0)
                     : launch_scat_gain<float>(dptr<float>(P->d_sig[l]) + o, dptr<float>(tmp) + o,
                                               reinterpret_cast<const Dir<float>*>(P->d_dir[l]), A.nd,
                                               (int)A.npix(), dptr<float>(P->d_scat_w[l]) + o, 0);
      }
      if (ge == cudaSuccess) ge = cudaStreamSynchronize(0);
      cudaFree(tmp);
      if (ge != cudaSuccess) return bail(fail(BTMG_ERR_CUDA, cudaGetErrorString(ge)));
      max_n = std::max(max_n, A.n());
      max_pix = std::max(max_pix, A.npix());
      max_part = std::max(max_part, (size_t)scat_chunks(A.nx, A.ny, A.nd, (int)P->csize) * A.npix());
      if (l == 0 && cudaMalloc(&P->d_delta[0], A.n() * P->csize) != cudaSuccess)
        return bail(fail(BTMG_ERR_OOM, "workspace delta"));
    }
    // the coarsest levels that fit the single-CTA tail kernel (not level 0)
    const int tmax = P->f64 ? scat_tail_max<double>() : scat_tail_max<float>();
    P->scat_tail = P->L;
    while (P->scat_tail - 1 >= 1 && P->L - (P->scat_tail - 1) <= kScatTailLevels && P->scat_on[P->scat_tail - 1] &&
           P->lev[P->scat_tail - 1].n() <= (size_t)tmax)
      --P->scat_tail;
    if (max_n && (cudaMalloc(&P->d_scat_j, max_n * P->csize) != cudaSuccess ||
                  cudaMalloc(&P->d_scat_part, max_part * P->csize) != cudaSuccess ||
                  cudaMalloc(&P->d_scat_c, max_pix * P->csize) != cudaSuccess))
      return bail(fail(BTMG_ERR_OOM, "scattering smoother workspace"));
  }
  if (P->f64) put_vals<double>(buf, sigs);
  else put_vals<float>(buf, sigs);
  if ((rc = upload(&P->d_sigs, buf))) return bail(rc);
  if (P->f64) put_vals<double>(buf, src);
  else put_vals<float>(buf, src);
  if ((rc = upload(&P->d_src, buf))) return bail(rc);
  if (cudaMalloc(&P->d_b, npix * P->csize) != cudaSuccess ||
      cudaMalloc(&P->d_phi_part, (size_t)G * P->nchunk * npix * P->csize) != cudaSuccess ||
      cudaMalloc(&P->d_psi_tmp, F.n() * dtype_size(P->dtype)) != cudaSuccess)
    return bail(fail(BTMG_ERR_OOM, "workspace"));
  convfem_stencils(d->order, P->st_m1, P->st_d1, P->st_s1);
  if (d->pg && d->order == 3 && cudaMalloc(&P->d_pgd, 4 * F.n() * P->csize) != cudaSuccess)
    return bail(fail(BTMG_ERR_OOM, "cubic PG scratch"));
  P->n_norm_sum = d->pg ? tiles * P->nchunk : upres_norm_blocks(F.nx, F.ny, P->nchunk);
  P->n_norm_part = std::max(tiles * P->nchunk, upres_norm_blocks(F.nx, F.ny, P->nchunk));
  P->n_q_blocks = (int)((npix + 255) / 256 < 1024 ? (npix + 255) / 256 : 1024);
  if (cudaMalloc(&P->d_norm_part, sizeof(double) * P->n_norm_part) != cudaSuccess ||
      cudaMalloc(&P->d_qn2_part, sizeof(double) * P->n_q_blocks) != cudaSuccess ||
      cudaMalloc(&P->d_rn2, sizeof(double) * G) != cudaSuccess ||
      cudaMalloc(&P->d_qn2, sizeof(double) * G) != cudaSuccess ||
      cudaMalloc(&P->d_err, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_pinned, sizeof(double) * (2 * G + 1)) != cudaSuccess)
    return bail(fail(BTMG_ERR_OOM, "workspace norms"));
  if (cudaStreamCreateWithFlags(&P->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->order_event, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(BTMG_ERR_CUDA, "stream creation"));
  cudaMemset(P->d_err, 0, sizeof(int));
  cudaMemset(P->d_rn2, 0, sizeof(double) * G);
  cudaMemset(P->d_qn2, 0, sizeof(double) * G);
  *out = P;
  return BTMG_OK;
}

int check_level(const btmg_problem* p, int level) {
  if (!p) return fail(BTMG_ERR_INVALID_ARG, "null problem");
  if (level < 0 || level >= p->L) return fail(BTMG_ERR_INVALID_ARG, "level out of range");
  return BTMG_OK;
}

// ------------------------------------------------------------ batches ----
// Whole cycle of one problem (scalar-flux partials and every group) captured
// as a graph on a non-default stream.
template <typename T, typename C> struct RunCapture {
  static int run(btmg_problem* P, void* psi, cudaStream_t s, cudaGraph_t* g) {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int rc = Impl<T, C>::mg_cycle(P, psi, nullptr, s);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CK(ee);
    *g = graph;
    return BTMG_OK;
  }
};
// relative residual of psi (all groups), FP64 norms
// The two parts of a one-group cycle around its coarse correction: A = the
// scalar-flux partials, source, fine residual and its norm; B = the finest
// level's sweeps from d_delta[1], source and fine PG Jacobi (the batched
// persistent launch does the levels in between).
template <typename T, typename C> struct RunCapturePart {
  static int run(btmg_problem* P, void* psi, int part, cudaStream_t s, cudaGraph_t* g) {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    T* ps = reinterpret_cast<T*>(psi);
    cudaError_t e = cudaSuccess;
    if (part == 0) {
      e = Impl<T, C>::phi_partials(P, ps, s);
      if (e == cudaSuccess) e = Impl<T, C>::cycle_part_a(P, ps, 0, s);
    } else {
      e = Impl<T, C>::cycle_part_b(P, ps, 0, s, false, true);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      CK(e != cudaSuccess ? e : ee);
    }
    *g = graph;
    return BTMG_OK;
  }
};

template <typename T, typename C> struct RunResidual {
  static int run(btmg_problem* P, const void* psi, double* rel, cudaStream_t s) {
    CK(Impl<T, C>::residual_all(P, reinterpret_cast<const T*>(psi), nullptr, s));
    return Impl<T, C>::read_rel(P, s, 0, nullptr, rel);
  }
};

// Particle balance of every group of psi (upwind fine scheme): production,
// removal, leakage and the relative imbalance, per group (k_balance.cu).
template <typename T, typename C> struct RunBalance {
  static int run(btmg_problem* P, const void* psi, double* out, cudaStream_t s) {
    const T* ps = reinterpret_cast<const T*>(psi);
    const LevelH& L0 = P->lev[0];
    const size_t npix = L0.npix();
    CK(Impl<T, C>::phi_partials(P, ps, s));
    const int nv = (int)std::min<size_t>(1024, (npix + 255) / 256);
    const int nl = (int)std::min<size_t>(1024, ((size_t)(L0.nx + L0.ny) * L0.nd + 255) / 256);
    double* part = nullptr;
    CK(cudaMalloc(&part, sizeof(double) * 2 * (nv + nl)));
    std::vector<double> h(2 * (nv + nl));
    const Bc bc{P->d.bc[0], P->d.bc[1], P->d.bc[2], P->d.bc[3]};
    int rc = BTMG_OK;
    for (int g = 0; g < P->G && rc == BTMG_OK; ++g) {
      cudaError_t e = launch_balance_volume<C>(dptr<C>(P->d_src) + g * npix, dptr<C>(P->d_sigs) + (size_t)g * P->G * npix,
                                               dptr<C>(P->d_sig[0]) + g * npix, dptr<C>(P->d_phi_part), P->G, g,
                                               P->nchunk, (int)npix, part, nv, s);
      if (e == cudaSuccess)
        e = launch_balance_leak<T, C>(ps + (size_t)g * L0.n(), reinterpret_cast<const Dir<C>*>(P->d_dir[0]), L0.nx,
                                      L0.ny, L0.nd, bc, L0.dx, L0.dy, part + 2 * nv, nl, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        rc = fail(BTMG_ERR_CUDA, cudaGetErrorString(e));
        break;
      }
      double prod = 0.0, rem = 0.0, leak = 0.0;
      for (int b = 0; b < nv; ++b) prod += h[2 * b], rem += h[2 * b + 1];
      for (int b = 0; b < nl; ++b) leak += h[2 * (nv + b)] + h[2 * (nv + b) + 1];
      prod *= L0.dx * L0.dy;
      rem *= L0.dx * L0.dy;
      out[4 * g + 0] = prod;
      out[4 * g + 1] = rem;
      out[4 * g + 2] = leak;
      out[4 * g + 3] = prod != 0.0 ? (prod - rem - leak) / prod : (prod - rem - leak);
    }
    cudaFree(part);
    return rc;
  }
};

// Autotuner cache: problem shape -> (chunks, ms per eager cycle).
struct TuneKey {
  int nx, ny, nd, G, dtype, pg, nu, scat;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nd, G, dtype, pg, nu, scat) <
           std::tie(o.nx, o.ny, o.nd, o.G, o.dtype, o.pg, o.nu, o.scat);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, double>> g_tune;

// Time `cycles` eager cycles (after `warm` untimed ones) of the problem d on s.
int time_cycles(const btmg_problem_desc& d, int warm, int cycles, cudaStream_t s, double* ms) {
  btmg_problem* P = nullptr;
  if (int rc = create(&d, &P)) return rc;
  void* psi = nullptr;
  const size_t bytes = (size_t)P->G * P->lev[0].n() * dtype_size(P->dtype);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BTMG_OK;
  auto done = [&](int code) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (psi) cudaFree(psi);
    destroy(P);
    return code;
  };
  if (cudaMalloc(&psi, bytes) != cudaSuccess) return done(fail(BTMG_ERR_OOM, "autotune: psi"));
  if (cudaMemsetAsync(psi, 0, bytes, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    return done(fail(BTMG_ERR_CUDA, "autotune: setup"));
  for (int k = 0; k < warm && rc == BTMG_OK; ++k) rc = dispatch<RunCycle>(P->dtype, P, psi, nullptr, s);
  if (rc) return done(rc);
  cudaEventRecord(e0, s);
  for (int k = 0; k < cycles && rc == BTMG_OK; ++k) rc = dispatch<RunCycle>(P->dtype, P, psi, nullptr, s);
  if (rc) return done(rc);
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) return done(fail(BTMG_ERR_CUDA, "autotune: timing"));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  *ms = t / cycles;
  return done(BTMG_OK);
}

// Chunk count for the shape of d: candidates are the divisors of the
// direction count (at most 64) within a factor 4 of the automatic choice,
// each timed over 3 eager cycles after 2 warm-up cycles.
int tune_chunks(const btmg_problem_desc& d, cudaStream_t s, int* chunks, double* ms) {
  const int nd = d.n_polar * d.n_azim;
  const int tiles = ((d.nx + kTile - 1) / kTile) * ((d.ny + kTile - 1) / kTile);
  const TuneKey key{d.nx, d.ny, nd, d.n_groups, d.psi_dtype, d.pg, d.nu_jacobi, d.scat_levels};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *chunks = it->second.first;
      *ms = it->second.second;
      return BTMG_OK;
    }
  }
  const int a = auto_chunks(d.psi_dtype, d.pg != 0, tiles, nd);
  int best = a;
  double best_ms = 1e300;
  for (int c = 1; c <= nd && c <= 64; ++c) {
    if (nd % c || 4 * c < a || c > 4 * a) continue;
    btmg_problem_desc d2 = d;
    d2.chunks = c;
    double t = 0.0;
    if (int rc = time_cycles(d2, 2, 3, s, &t)) return rc;
    if (t < best_ms) {
      best_ms = t;
      best = c;
    }
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {best, best_ms};
  *chunks = best;
  *ms = best_ms;
  return BTMG_OK;
}

}  // namespace

struct btmg_batch {
  std::vector<btmg_problem*> probs;
  std::vector<int> auto_ch;
  std::vector<double> tuned_ms;
  cudaStream_t bs = nullptr;    // capture and launch stream
  cudaEvent_t order = nullptr;  // orders bs after the caller's stream and back
  std::vector<cudaGraph_t> cyc;  // per problem: one whole cycle
  std::vector<const void*> cyc_psi;
  cudaGraphExec_t exec = nullptr;  // parent graph of the active problems
  std::vector<int> exec_set;
  double* h_res = nullptr;  // pinned: per problem rn2[G], qn2[G]
  int* h_err = nullptr;     // pinned: per problem bounded-wait flag
  std::vector<size_t> res_off;
  // persistent coarse correction (one-group problems with FP32 compute): the
  // cycle of every active problem is part A (fine residual), one persistent
  // launch of every problem's restrictions and coarse sweeps, part B (finest
  // sweeps and PG Jacobi)
  bool persist = false;
  bool autotune = false, tuned = false;
  int tu = 32, ctas = 2;           // sweep tile width and CTAs per SM of the launch
  double coarse_ms = 0.0;          // tuned time of one persistent launch
  std::vector<cudaGraph_t> cycA, cycB;
  cudaGraph_t coarse = nullptr;    // counter reset + persistent launch, active set
  void* d_plan = nullptr;          // segments, tasks and arguments of the active set
  unsigned* d_cnt = nullptr;       // head + done per segment
  int* d_cerr = nullptr;           // bounded-wait flag of the persistent launch
  int* h_cerr = nullptr;           // pinned copy
  size_t cnt_cap = 0, plan_cap = 0;
};

namespace {
void batch_free(btmg_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (cudaGraph_t g : B->cyc)
    if (g) cudaGraphDestroy(g);
  for (cudaGraph_t g : B->cycA)
    if (g) cudaGraphDestroy(g);
  for (cudaGraph_t g : B->cycB)
    if (g) cudaGraphDestroy(g);
  if (B->coarse) cudaGraphDestroy(B->coarse);
  if (B->d_plan) cudaFree(B->d_plan);
  if (B->d_cnt) cudaFree(B->d_cnt);
  if (B->d_cerr) cudaFree(B->d_cerr);
  if (B->h_cerr) cudaFreeHost(B->h_cerr);
  for (btmg_problem* P : B->probs) destroy(P);
  if (B->h_res) cudaFreeHost(B->h_res);
  if (B->h_err) cudaFreeHost(B->h_err);
  if (B->order) cudaEventDestroy(B->order);
  if (B->bs) cudaStreamDestroy(B->bs);
  delete B;
}

// The coarse correction of a one-group problem as segments of the persistent
// batched launch, in the order of cycle_part_b: the restrictions down every
// level (Sec. 2.5), then the nu upwind Jacobi sweeps from the coarsest level
// up to level 1 (Eq. matrix_full, beta = 1; UpSamp of the coarser level's
// correction), each segment waiting for the one before it.  FP32 compute.
void coarse_plan(btmg_problem* P, int tu, std::vector<CoarseSeg>& segs, std::vector<CoarseRestrict>& ra,
                 std::vector<UpArgs<float, float>>& ua) {
  const int L = P->L;
  int prev = -1;
  for (int l = 0; l + 1 < L; ++l) {
    const LevelH &A = P->lev[l], &B = P->lev[l + 1];
    ra.push_back(CoarseRestrict{dptr<float>(P->d_s[l]), dptr<float>(P->d_s[l + 1]), dptr<float>(P->d_rcoef[l]), A.nx,
                                A.ny, A.nr, A.nc, B.nx, B.ny, B.nr, B.nc, A.fx, A.fy, A.fr, A.fc});
    segs.push_back(CoarseSeg{0, (int)ra.size() - 1, (int)((B.n() + kCoarseCells - 1) / kCoarseCells), prev, 0});
    prev = (int)segs.size() - 1;
  }
  for (int l = L - 1; l >= 1; --l) {
    const LevelH& A = P->lev[l];
    UpArgs<float, float> u{};
    u.sig = dptr<float>(P->d_sig[l]);
    u.dir = reinterpret_cast<const Dir<float>*>(P->d_dir[l]);
    u.nx = A.nx;
    u.ny = A.ny;
    u.nr = A.nr;
    u.nc = A.nc;
    u.nd = A.nd;
    u.nu = P->d.nu_jacobi;
    u.src_stride = A.npix();
    u.tiles_x = (A.nx + tu - 1) / tu;
    u.bc = Bc{P->d.bc[0], P->d.bc[1], P->d.bc[2], P->d.bc[3]};
    u.dpc = 1;
    u.err = P->d_err;
    u.src = dptr<float>(P->d_s[l]);
    u.delta_out = dptr<float>(P->d_delta[l]);
    u.init_mode = l == L - 1 ? INIT_ZERO : INIT_UPSAMPLE;
    if (l + 1 < L) {
      const LevelH& B = P->lev[l + 1];
      u.init = dptr<float>(P->d_delta[l + 1]);
      u.nxc = B.nx;
      u.nyc = B.ny;
      u.nrc = B.nr;
      u.ncc = B.nc;
      u.fx = A.fx;
      u.fy = A.fy;
      u.fr = A.fr;
      u.fc = A.fc;
      u.parent = reinterpret_cast<const int*>(P->d_parent[l]);
    }
    ua.push_back(u);
    const int tiles = u.tiles_x * ((A.ny + tu - 1) / tu);
    segs.push_back(CoarseSeg{1, (int)ua.size() - 1, tiles * A.nd, prev, tiles});
    prev = (int)segs.size() - 1;
  }
}

// Builds (on B->bs, by stream capture) the graph of one persistent coarse
// launch over the active problems with tile width tu and ctas CTAs per SM:
// the task plan is uploaded, the counters and the error word are zeroed,
// then the kernel drains the queue.  Tasks are ordered by the index of their
// segment inside its problem's chain, then by problem and block, so every
// prerequisite precedes its dependents.
int coarse_graph(btmg_batch* B, const std::vector<int>& active, int tu, int ctas, cudaGraph_t* out) {
  std::vector<CoarseSeg> segs;
  std::vector<CoarseRestrict> ra;
  std::vector<UpArgs<float, float>> ua;
  std::vector<int> first(active.size() + 1, 0);
  for (size_t k = 0; k < active.size(); ++k) {
    first[k] = (int)segs.size();
    coarse_plan(B->probs[active[k]], tu, segs, ra, ua);
  }
  first[active.size()] = (int)segs.size();
  std::vector<int2> tasks;
  for (int stage = 0;; ++stage) {
    bool any = false;
    for (size_t k = 0; k < active.size(); ++k) {
      const int sg = first[k] + stage;
      if (sg >= first[k + 1]) continue;
      any = true;
      for (int b = 0; b < segs[sg].blocks; ++b) tasks.push_back(make_int2(sg, b));
    }
    if (!any) break;
  }
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t o_task = al(segs.size() * sizeof(CoarseSeg)), o_ra = o_task + al(tasks.size() * sizeof(int2));
  const size_t o_ua = o_ra + al(ra.size() * sizeof(CoarseRestrict)), bytes = o_ua + al(ua.size() * sizeof(UpArgs<float, float>));
  if (bytes > B->plan_cap) {
    if (B->d_plan) cudaFree(B->d_plan);
    B->d_plan = nullptr;
    B->plan_cap = 0;
    if (cudaMalloc(&B->d_plan, bytes) != cudaSuccess) return fail(BTMG_ERR_OOM, "batch plan");
    B->plan_cap = bytes;
  }
  if (1 + segs.size() > B->cnt_cap) {
    if (B->d_cnt) cudaFree(B->d_cnt);
    B->d_cnt = nullptr;
    B->cnt_cap = 0;
    if (cudaMalloc(&B->d_cnt, (1 + segs.size()) * sizeof(unsigned)) != cudaSuccess)
      return fail(BTMG_ERR_OOM, "batch counters");
    B->cnt_cap = 1 + segs.size();
  }
  char* base = static_cast<char*>(B->d_plan);
  std::vector<char> host(bytes, 0);
  memcpy(host.data(), segs.data(), segs.size() * sizeof(CoarseSeg));
  memcpy(host.data() + o_task, tasks.data(), tasks.size() * sizeof(int2));
  memcpy(host.data() + o_ra, ra.data(), ra.size() * sizeof(CoarseRestrict));
  memcpy(host.data() + o_ua, ua.data(), ua.size() * sizeof(UpArgs<float, float>));
  CK(cudaMemcpyAsync(B->d_plan, host.data(), bytes, cudaMemcpyHostToDevice, B->bs));
  CK(cudaStreamSynchronize(B->bs));
  CoarseBatch cb{};
  cb.seg = reinterpret_cast<const CoarseSeg*>(base);
  cb.task = reinterpret_cast<const int2*>(base + o_task);
  cb.ntasks = (int)tasks.size();
  cb.ra = reinterpret_cast<const CoarseRestrict*>(base + o_ra);
  cb.ua = reinterpret_cast<const UpArgs<float, float>*>(base + o_ua);
  cb.head = B->d_cnt;
  cb.done = B->d_cnt + 1;
  cb.err = B->d_cerr;
  const int nu = B->probs[active[0]]->d.nu_jacobi;
  CK(cudaStreamBeginCapture(B->bs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(B->d_cnt, 0, (1 + segs.size()) * sizeof(unsigned), B->bs);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_cerr, 0, sizeof(int), B->bs);
  if (e == cudaSuccess && cb.ntasks > 0) e = launch_coarse_batch(cb, nu, tu, ctas, B->bs);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(B->bs, &g);
  if (e != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    CK(e != cudaSuccess ? e : ee);
  }
  *out = g;
  return BTMG_OK;
}

// The tile width and grid of the persistent launch, timed: each candidate's
// graph runs 2 warm-up and 5 timed times (CUDA events on B->bs) on the
// current restricted residuals (the launch only rewrites the coarse levels,
// which the next cycle recomputes); the fastest is kept.
int coarse_tune(btmg_batch* B, const std::vector<int>& active) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int best_tu = B->tu, best_ctas = B->ctas;
  for (int tu : {16, 32})
    for (int ctas : {1, 2, 4}) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t x = nullptr;
      if (int rc = coarse_graph(B, active, tu, ctas, &g)) return rc;
      cudaError_t e = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      CK(e);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaGraphLaunch(x, B->bs);
      if (e == cudaSuccess) e = cudaEventRecord(e0, B->bs);
      for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaGraphLaunch(x, B->bs);
      if (e == cudaSuccess) e = cudaEventRecord(e1, B->bs);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      cudaGraphExecDestroy(x);
      CK(e);
      if (ms / 5 < best) {
        best = ms / 5;
        best_tu = tu;
        best_ctas = ctas;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->tu = best_tu;
  B->ctas = best_ctas;
  B->coarse_ms = best;
  B->tuned = true;
  return BTMG_OK;
}

// persistent form of the parent graph: every active problem's part A, then
// the persistent coarse launch of all of them, then every problem's part B
// followed by the copies of its residual norms and error flag
int batch_build_persistent(btmg_batch* B, const std::vector<int>& active) {
  if (B->coarse) cudaGraphDestroy(B->coarse);
  B->coarse = nullptr;
  if (int rc = coarse_graph(B, active, B->tu, B->ctas, &B->coarse)) return rc;
  cudaGraph_t parent = nullptr;
  CK(cudaGraphCreate(&parent, 0));
  std::vector<cudaGraphNode_t> as;
  cudaError_t e = cudaSuccess;
  for (int i : active) {
    cudaGraphNode_t a;
    if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&a, parent, nullptr, 0, B->cycA[i]);
    as.push_back(a);
  }
  cudaGraphNode_t cn, cm;
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&cn, parent, as.data(), as.size(), B->coarse);
  if (e == cudaSuccess)
    e = cudaGraphAddMemcpyNode1D(&cm, parent, &cn, 1, B->h_cerr, B->d_cerr, sizeof(int), cudaMemcpyDeviceToHost);
  for (int i : active) {
    btmg_problem* P = B->probs[i];
    cudaGraphNode_t child, m0, m1, m2;
    if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, parent, &cn, 1, B->cycB[i]);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&m0, parent, &child, 1, B->h_res + B->res_off[i], P->d_rn2,
                                   sizeof(double) * P->G, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&m1, parent, &child, 1, B->h_res + B->res_off[i] + P->G, P->d_qn2,
                                   sizeof(double) * P->G, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&m2, parent, &child, 1, B->h_err + i, P->d_err, sizeof(int),
                                   cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(parent);
    CK(e);
  }
  const cudaError_t ei = cudaGraphInstantiate(&B->exec, parent, 0);
  cudaGraphDestroy(parent);
  CK(ei);
  B->exec_set = active;
  return BTMG_OK;
}

// parent graph: one child-graph branch per active problem, each followed by
// the copies of its residual norms and its error flag to pinned host memory
int batch_build(btmg_batch* B, const std::vector<int>& active) {
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  cudaGraph_t parent = nullptr;
  CK(cudaGraphCreate(&parent, 0));
  for (int i : active) {
    btmg_problem* P = B->probs[i];
    cudaGraphNode_t child, m0, m1, m2;
    cudaError_t e = cudaGraphAddChildGraphNode(&child, parent, nullptr, 0, B->cyc[i]);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&m0, parent, &child, 1, B->h_res + B->res_off[i], P->d_rn2,
                                   sizeof(double) * P->G, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&m1, parent, &child, 1, B->h_res + B->res_off[i] + P->G, P->d_qn2,
                                   sizeof(double) * P->G, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&m2, parent, &child, 1, B->h_err + i, P->d_err, sizeof(int),
                                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaGraphDestroy(parent);
      CK(e);
    }
  }
  const cudaError_t ei = cudaGraphInstantiate(&B->exec, parent, 0);
  cudaGraphDestroy(parent);
  CK(ei);
  B->exec_set = active;
  return BTMG_OK;
}

int solve_batch(btmg_batch* B, void* const* psi, double rtol, int max_cycles, int check, btmg_solve_info* infos,
                cudaStream_t s) {
  const int n = (int)B->probs.size();
  CK(cudaEventRecord(B->order, s));
  CK(cudaStreamWaitEvent(B->bs, B->order, 0));
  std::vector<int> cycles(n, 0), status(n, BTMG_ERR_NOT_CONVERGED);
  std::vector<double> best(n, 1e300), rel(n, 0.0);
  std::vector<char> done(n, 0);
  // first cycle eagerly (kernel attributes, workspaces), then capture
  bool recaptured = false;
  for (int i = 0; i < n; ++i) {
    btmg_problem* P = B->probs[i];
    if (int rc = dispatch<RunCycle>(P->dtype, P, psi[i], nullptr, B->bs)) return rc;
    cycles[i] = 1;
    if (!B->cyc[i] || B->cyc_psi[i] != psi[i]) {
      if (B->cyc[i]) cudaGraphDestroy(B->cyc[i]);
      B->cyc[i] = nullptr;
      if (int rc = dispatch<RunCapture>(P->dtype, P, psi[i], B->bs, &B->cyc[i])) return rc;
      B->cyc_psi[i] = psi[i];
      recaptured = true;
    }
    if (cycles[i] >= max_cycles) done[i] = 1;
  }
  if (recaptured && B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  if (B->persist) {  // the two parts of every cycle, and the launch's tuning
    for (int i = 0; i < n; ++i) {
      btmg_problem* P = B->probs[i];
      if (!B->cycA[i] || recaptured) {
        for (cudaGraph_t* gp : {&B->cycA[i], &B->cycB[i]}) {
          if (*gp) cudaGraphDestroy(*gp);
          *gp = nullptr;
        }
        if (int rc = dispatch<RunCapturePart>(P->dtype, P, psi[i], 0, B->bs, &B->cycA[i])) return rc;
        if (int rc = dispatch<RunCapturePart>(P->dtype, P, psi[i], 1, B->bs, &B->cycB[i])) return rc;
      }
    }
    if (B->autotune && !B->tuned) {
      std::vector<int> all(n);
      for (int i = 0; i < n; ++i) all[i] = i;
      if (int rc = coarse_tune(B, all)) return rc;
      if (B->exec) cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
    }
  }
  const double pi4 = 4.0 * kPi;
  for (;;) {
    std::vector<int> active;
    int k = check;
    for (int i = 0; i < n; ++i)
      if (!done[i]) {
        active.push_back(i);
        k = std::min(k, max_cycles - cycles[i]);
      }
    if (active.empty()) break;
    if (!B->exec || active != B->exec_set) {
      if (B->exec) cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
      if (int rc = B->persist ? batch_build_persistent(B, active) : batch_build(B, active)) return rc;
    }
    for (int j = 0; j < k; ++j) CK(cudaGraphLaunch(B->exec, B->bs));
    CK(cudaStreamSynchronize(B->bs));
    if (B->persist && *B->h_cerr) return fail(BTMG_ERR_TIMEOUT, "a bounded device wait gave up (persistent launch)");
    for (int i : active) {
      btmg_problem* P = B->probs[i];
      cycles[i] += k;
      if (B->h_err[i]) return fail(BTMG_ERR_TIMEOUT, "a bounded device wait gave up (batch problem)");
      double sr = 0.0, sq = 0.0;
      for (int g = 0; g < P->G; ++g) {
        sr += B->h_res[B->res_off[i] + g];
        sq += B->h_res[B->res_off[i] + P->G + g];
      }
      const double w = pi4 * P->lev[0].dx * P->lev[0].dy;
      const double r = sq > 0 ? std::sqrt(sr / (w * sq)) : std::sqrt(sr);
      if (std::isnan(r)) {
        status[i] = BTMG_ERR_NAN;
        done[i] = 1;
      } else if (r > 1e3 * best[i] && best[i] < 1e299) {
        status[i] = BTMG_ERR_DIVERGED;
        done[i] = 1;
      } else {
        best[i] = std::min(best[i], r);
        if (r <= rtol) {
          status[i] = BTMG_OK;
          done[i] = 1;
        } else if (cycles[i] >= max_cycles) {
          done[i] = 1;
        }
      }
    }
  }
  // residual of every returned psi (FP64 norms)
  int result = BTMG_OK;
  for (int i = 0; i < n; ++i) {
    btmg_problem* P = B->probs[i];
    if (int rc = dispatch<RunResidual>(P->dtype, P, (const void*)psi[i], &rel[i], B->bs)) return rc;
    if (status[i] == BTMG_OK && !(rel[i] <= rtol))
      status[i] = std::isnan(rel[i]) ? BTMG_ERR_NAN : BTMG_ERR_NOT_CONVERGED;
    if (infos) {
      infos[i].cycles = cycles[i];
      infos[i].status = status[i];
      infos[i].rel_resid = rel[i];
    }
    if (status[i] != BTMG_OK && result == BTMG_OK) result = BTMG_ERR_NOT_CONVERGED;
  }
  CK(cudaEventRecord(B->order, B->bs));
  CK(cudaStreamWaitEvent(s, B->order, 0));
  return result;
}
}  // namespace

namespace {
// FP32 FMA throughput probe: kFmaChains independent FFMA chains per thread
// (enough to cover the pipe latency), iters rounds; the result is written
// only under a condition the compiler cannot decide, so no chain is removed.
constexpr int kFmaChains = 8;
__global__ void k_fma_probe(float* out, int iters) {
  float v[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) v[k] = 1e-3f * (float)(threadIdx.x + k);
  const float m = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) v[k] = fmaf(v[k], m, c);
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) sum += v[k];
  if (sum == -1.0f) out[0] = sum;
}
cudaError_t launch_fma_probe(float* out, int iters, int blocks, int block, cudaStream_t s) {
  k_fma_probe<<<blocks, block, 0, s>>>(out, iters);
  return cudaGetLastError();
}
}  // namespace

extern "C" {

int btmg_create_problem(const btmg_problem_desc* desc, void* stream, btmg_problem** out) {
  (void)stream;
  try {
    return create(desc, out);
  } catch (...) {
    return fail(BTMG_ERR_OOM, "host allocation failed");
  }
}

int btmg_destroy_problem(btmg_problem* p) {
  destroy(p);
  return BTMG_OK;
}

int btmg_num_unknowns(const btmg_problem* p, int64_t* n) {
  if (!p || !n) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  *n = (int64_t)p->G * (int64_t)p->lev[0].n();
  return BTMG_OK;
}

int btmg_get_layout(const btmg_problem* p, int64_t strides[6]) {
  if (!p || !strides) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  const LevelH& A = p->lev[0];
  strides[5] = 1;
  strides[4] = A.nx;
  strides[3] = (int64_t)A.nx * A.ny;
  strides[2] = strides[3] * A.nc;
  strides[1] = strides[2] * A.nr;
  strides[0] = strides[1] * 8;
  return BTMG_OK;
}

int btmg_num_levels(const btmg_problem* p, int32_t* levels) {
  if (!p || !levels) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  *levels = p->L;
  return BTMG_OK;
}

int btmg_level_info(const btmg_problem* p, int32_t level, int32_t dims[5], double dxdy[2]) {
  if (int rc = check_level(p, level)) return rc;
  const LevelH& A = p->lev[level];
  if (dims) {
    dims[0] = A.nx;
    dims[1] = A.ny;
    dims[2] = A.nr;
    dims[3] = A.nc;
    dims[4] = A.nd;
  }
  if (dxdy) {
    dxdy[0] = A.dx;
    dxdy[1] = A.dy;
  }
  return BTMG_OK;
}

int btmg_level_quadrature(const btmg_problem* p, int32_t level, double* mu, double* nu, double* w) {
  if (int rc = check_level(p, level)) return rc;
  const LevelH& A = p->lev[level];
  for (int n = 0; n < A.nd; ++n) {
    if (mu) mu[n] = A.mu[n];
    if (nu) nu[n] = A.nu[n];
    if (w) w[n] = A.p[n];
  }
  return BTMG_OK;
}

int btmg_scalar_flux(btmg_problem* p, const void* psi, void* phi, void* stream) {
  if (!p || !psi || !phi) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  return dispatch<RunFlux>(p->dtype, p, psi, phi, (cudaStream_t)stream);
}

int btmg_apply_operator(btmg_problem* p, const void* psi, void* r, void* stream) {
  if (!p || !psi || !r) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  return dispatch<RunApply>(p->dtype, p, psi, r, (cudaStream_t)stream);
}

int btmg_smooth(btmg_problem* p, void* psi, const void* src, int32_t level, int32_t group, int32_t sweeps,
                int32_t kind, void* stream) {
  if (int rc = check_level(p, level)) return rc;
  if (!psi || sweeps < 0) return fail(BTMG_ERR_INVALID_ARG, "bad psi or sweeps");
  if (kind == BTMG_SMOOTH_PG) {
    if (level != 0 || src) return fail(BTMG_ERR_INVALID_ARG, "PG smoothing is on level 0 with src = NULL");
    return dispatch<RunSmoothPG>(p->dtype, p, psi, (int)sweeps, (cudaStream_t)stream);
  }
  if (kind != BTMG_SMOOTH_UPWIND) return fail(BTMG_ERR_INVALID_ARG, "bad smoother kind");
  if (!src || group < 0 || group >= p->G) return fail(BTMG_ERR_INVALID_ARG, "upwind smoothing needs src and group");
  return dispatch<RunSmoothUp>(p->dtype, p, psi, src, (int)level, (int)group, (int)sweeps, (cudaStream_t)stream);
}

int btmg_restrict(btmg_problem* p, int32_t level, const void* fine, void* coarse, void* stream) {
  if (int rc = check_level(p, level)) return rc;
  if (level + 1 >= p->L || !fine || !coarse) return fail(BTMG_ERR_INVALID_ARG, "bad restriction arguments");
  const LevelH &A = p->lev[level], &B = p->lev[level + 1];
  cudaError_t e = p->f64 ? launch_restrict<double>((const double*)fine, (double*)coarse, (const double*)p->d_rcoef[level], A.nx,
                                                   A.ny, A.nr, A.nc, B.nx, B.ny, B.nr, B.nc, A.fx, A.fy, A.fr, A.fc,
                                                   (cudaStream_t)stream)
                         : launch_restrict<float>((const float*)fine, (float*)coarse, (const float*)p->d_rcoef[level], A.nx,
                                                  A.ny, A.nr, A.nc, B.nx, B.ny, B.nr, B.nc, A.fx, A.fy, A.fr, A.fc,
                                                  (cudaStream_t)stream);
  CK(e);
  return BTMG_OK;
}

int btmg_prolong(btmg_problem* p, int32_t level, const void* coarse, void* fine, void* stream) {
  if (int rc = check_level(p, level)) return rc;
  if (level + 1 >= p->L || !fine || !coarse) return fail(BTMG_ERR_INVALID_ARG, "bad prolongation arguments");
  const LevelH &A = p->lev[level], &B = p->lev[level + 1];
  cudaError_t e = p->f64 ? launch_prolong<double>((const double*)coarse, (double*)fine, A.nx, A.ny, A.nr, A.nc, B.nx,
                                                  B.ny, B.nr, B.nc, A.fx, A.fy, A.fr, A.fc, (cudaStream_t)stream)
                         : launch_prolong<float>((const float*)coarse, (float*)fine, A.nx, A.ny, A.nr, A.nc, B.nx,
                                                 B.ny, B.nr, B.nc, A.fx, A.fy, A.fr, A.fc, (cudaStream_t)stream);
  CK(e);
  return BTMG_OK;
}

int btmg_mg_cycle(btmg_problem* p, void* psi, double* rel_resid, void* stream) {
  if (!p || !psi) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  return dispatch<RunCycle>(p->dtype, p, psi, rel_resid, (cudaStream_t)stream);
}

int btmg_mg_cycle_host(btmg_problem* p, const void* psi_in, void* psi_out, double* rel_resid, void* stream) {
  if (!p || !psi_in || !psi_out) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  return dispatch<RunCycleHost>(p->dtype, p, psi_in, psi_out, rel_resid, (cudaStream_t)stream);
}

int btmg_solve(btmg_problem* p, void* psi, double rtol, int32_t max_cycles, btmg_solve_info* info, void* stream) {
  if (!p || !psi || max_cycles < 1) return fail(BTMG_ERR_INVALID_ARG, "bad solve arguments");
  return dispatch<RunSolve>(p->dtype, p, psi, rtol, (int)max_cycles, info, (cudaStream_t)stream);
}

namespace {
// Coarse canvas of the learned correction: factor f = ceil(max(nx, ny) / 64),
// canvas ceil(n / f) rounded up to a multiple of 8 (the U-net pools 3 times).
void learn_canvas(int nx, int ny, int* f, int* h8, int* w8) {
  const int m = std::max(nx, ny);
  *f = std::max(1, (m + 63) / 64);
  *w8 = std::max(8, ((nx + *f - 1) / *f + 7) / 8 * 8);
  *h8 = std::max(8, ((ny + *f - 1) / *f + 7) / 8 * 8);
}

int ensure_learn_ws(btmg_problem* P) {
  if (P->d_rho_part) return BTMG_OK;
  const LevelH& L0 = P->lev[0];
  learn_canvas(L0.nx, L0.ny, &P->lf, &P->H8, &P->W8);
  const size_t es = dtype_size(P->dtype);
  CK(cudaMalloc(&P->d_rho_part, (size_t)P->G * P->nchunk * L0.npix() * P->csize));
  CK(cudaMalloc(&P->d_feat, sizeof(float) * kLearnFeatures * P->H8 * P->W8));
  CK(cudaMalloc(&P->d_dimg, sizeof(float) * P->H8 * P->W8));
  CK(cudaMalloc(&P->d_lscale, sizeof(float)));
  CK(cudaMalloc(&P->d_lsum, sizeof(double) * 2));
  // partial sums of the canvas features and of the correction's source norm
  CK(cudaMalloc(&P->d_lpart, sizeof(double) * std::max(2 * kLearnBlocks, P->n_q_blocks)));
  CK(cudaMalloc(&P->d_lc, L0.n() * es));
  CK(cudaMalloc(&P->d_lr, L0.n() * P->csize));
  CK(cudaMalloc(&P->d_lb, L0.npix() * P->csize));
  CK(cudaMalloc(&P->d_ldot, sizeof(double) * 4));
  CK(cudaMalloc(&P->d_ldpart, sizeof(double) * kDotBlocks));
  CK(cudaMalloc(&P->d_lstat, sizeof(double) * 3));
  CK(cudaMalloc(&P->d_lphi, (size_t)P->nchunk * L0.npix() * P->csize));
  CK(cudaMalloc(&P->d_lzero, L0.npix() * P->csize));
  CK(cudaMalloc(&P->d_lphi0, L0.npix() * P->csize));
  CK(cudaMalloc(&P->d_lprev_all, (size_t)P->G * L0.npix() * P->csize));
  CK(cudaMemset(P->d_lzero, 0, L0.npix() * P->csize));
  CK(cudaMemset(P->d_lstat, 0, sizeof(double) * 3));
  return BTMG_OK;
}
}  // namespace

int btmg_set_learned(btmg_problem* p, btmg_unet* unet, int32_t every) {
  if (!p || every < 1) return fail(BTMG_ERR_INVALID_ARG, "bad learned-correction arguments");
  if (unet) {
    if (unet_in_channels(unet) != kLearnFeatures)
      return fail(BTMG_ERR_INVALID_ARG, "the learned correction needs a U-net with 4 input channels");
    if (int rc = ensure_learn_ws(p)) return rc;
  }
  free_graphs(p);
  p->learned = unet;
  p->learn_every = every;
  p->learn_count = 0;
  p->learn_fallbacks = 0;
  if (p->d_lstat) CK(cudaMemset(p->d_lstat, 0, sizeof(double) * 3));
  return BTMG_OK;
}

int btmg_particle_balance(btmg_problem* p, const void* psi, double* out, void* stream) {
  if (!p || !psi || !out) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  if (p->d.pg) return fail(BTMG_ERR_UNSUPPORTED, "the particle balance is that of the upwind fine scheme (pg = 0)");
  return dispatch<RunBalance>(p->dtype, p, psi, out, (cudaStream_t)stream);
}

int btmg_convfem_stencils(int32_t order, double* m1, double* d1, double* s1) {
  if (order < 1 || order > 3 || !m1 || !d1 || !s1) return fail(BTMG_ERR_INVALID_ARG, "bad order or NULL output");
  convfem_stencils(order, m1, d1, s1);
  return BTMG_OK;
}

int btmg_scatter_fallbacks(const btmg_problem* p, int32_t* fallbacks) {
  if (!p || !fallbacks) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  *fallbacks = p->scat_fallbacks;
  return BTMG_OK;
}

int btmg_learn_stats(btmg_problem* p, int64_t* steps, double* mean_factor, double* last_alpha,
                     int32_t* fallbacks) {
  if (!p) return fail(BTMG_ERR_INVALID_ARG, "null problem");
  double st[3] = {0.0, 0.0, 0.0};
  if (p->d_lstat) {
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(st, p->d_lstat, sizeof st, cudaMemcpyDeviceToHost));
  }
  if (steps) *steps = (int64_t)st[1];
  if (mean_factor) *mean_factor = st[1] > 0 ? st[0] / st[1] : 0.0;
  if (last_alpha) *last_alpha = st[2];
  if (fallbacks) *fallbacks = p->learn_fallbacks;
  return BTMG_OK;
}

int btmg_learn_canvas(const btmg_problem* p, int32_t* h8, int32_t* w8, int32_t* factor) {
  if (!p) return fail(BTMG_ERR_INVALID_ARG, "null problem");
  int f, h, w;
  learn_canvas(p->lev[0].nx, p->lev[0].ny, &f, &h, &w);
  if (h8) *h8 = h;
  if (w8) *w8 = w;
  if (factor) *factor = f;
  return BTMG_OK;
}

int btmg_learn_features(btmg_problem* p, const void* psi, const void* psi_prev, float* feat, float* scale,
                        void* stream) {
  if (!p || !psi || !feat || !scale) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  if (int rc = ensure_learn_ws(p)) return rc;
  return dispatch<RunFeatures>(p->dtype, p, psi, psi_prev, feat, scale, (cudaStream_t)stream);
}

int btmg_solve_refined(btmg_problem* p, double* psi64, double rtol, int32_t max_outer, int32_t inner_cycles,
                       btmg_solve_info* info, void* stream) {
  if (!p || !psi64 || max_outer < 0 || inner_cycles < 1) return fail(BTMG_ERR_INVALID_ARG, "bad refinement arguments");
  if (p->d.pg) return fail(BTMG_ERR_UNSUPPORTED, "refinement needs the linear (pg = 0) fine operator");
  cudaStream_t s = (cudaStream_t)stream;
  return dispatch<RunRefine>(p->dtype, p, psi64, rtol, (int)max_outer, (int)inner_cycles, info, s);
}

int btmg_profile(btmg_problem* p, int32_t enable) {
  if (!p) return fail(BTMG_ERR_INVALID_ARG, "null problem");
  p->prof_on = enable != 0;
  p->prof_cls.clear();
  return BTMG_OK;
}

int btmg_profile_read(btmg_problem* p, double* ms, int64_t* count, int32_t n_classes) {
  if (!p || !ms || !count || n_classes < 1) return fail(BTMG_ERR_INVALID_ARG, "bad profile arguments");
  for (int c = 0; c < n_classes; ++c) {
    ms[c] = 0.0;
    count[c] = 0;
  }
  for (size_t i = 0; i < p->prof_cls.size(); ++i) {
    CK(cudaEventSynchronize(p->prof_pool[2 * i + 1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p->prof_pool[2 * i], p->prof_pool[2 * i + 1]));
    const int c = p->prof_cls[i];
    if (c < n_classes) {
      ms[c] += t;
      count[c] += 1;
    }
  }
  p->prof_cls.clear();
  return BTMG_OK;
}

int btmg_launch_count(const btmg_problem* p, int64_t* n) {
  if (!p || !n) return fail(BTMG_ERR_INVALID_ARG, "null argument");
  *n = p->launches;
  return BTMG_OK;
}

const char* btmg_error_string(int status) {
  switch (status) {
    case BTMG_OK: return "ok";
    case BTMG_ERR_INVALID_ARG: return "invalid argument";
    case BTMG_ERR_CUDA: return "CUDA error";
    case BTMG_ERR_OOM: return "out of memory";
    case BTMG_ERR_NOT_CONVERGED: return "not converged";
    case BTMG_ERR_DIVERGED: return "diverged";
    case BTMG_ERR_TIMEOUT: return "timeout";
    case BTMG_ERR_NAN: return "NaN in the iteration";
    case BTMG_ERR_UNSUPPORTED: return "unsupported configuration";
    case BTMG_ERR_NOALLOC_TOO_LARGE: return "size beyond the allocation-free maximum";
  }
  return "unknown status";
}

const char* btmg_last_error(void) { return g_last_error.c_str(); }

int btmg_fp32_fma_rate(int32_t repeats, double* tflops, void* stream) {
  if (repeats < 1 || !tflops) return fail(BTMG_ERR_INVALID_ARG, "bad FMA-rate arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 152, threads = 2048;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
  const int block = 256, blocks = sms * (threads / block), iters = 1 << 15;
  float* d = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaMalloc(&d, sizeof(float)));
  double best = 0.0;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_fma_probe(d, iters, blocks, block, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kFmaChains * (double)iters * blocks * block;
    if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  CK(e);
  *tflops = best;
  return BTMG_OK;
}

int btmg_wait_selftest(int32_t polls, void* stream) {
  if (polls < 1) return fail(BTMG_ERR_INVALID_ARG, "polls must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  int h = 0;
  CK(cudaMalloc(&d, sizeof(int)));
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_wait_selftest(d, polls, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  CK(e);
  return h ? fail(BTMG_ERR_TIMEOUT, "bounded wait gave up (self-test)") : BTMG_OK;
}

int btmg_create_batch(const btmg_problem_desc* descs, int32_t n, int32_t autotune, void* stream,
                      btmg_batch** out) {
  if (!descs || n < 1 || !out) return fail(BTMG_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  btmg_batch* B = nullptr;
  try {
    B = new btmg_batch();
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&B->bs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->order, cudaEventDisableTiming) != cudaSuccess) {
      batch_free(B);
      return fail(BTMG_ERR_CUDA, "batch stream");
    }
    if (!s) s = B->bs;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
      btmg_problem_desc d = descs[i];
      const int nd = d.n_polar * d.n_azim;
      const int tiles = ((d.nx + kTile - 1) / kTile) * ((d.ny + kTile - 1) / kTile);
      double ms = 0.0;
      if (autotune && d.chunks == 0 && d.nx > 0 && d.ny > 0 && d.n_polar > 0 && d.n_azim > 0) {
        int c = 0;
        if (int rc = tune_chunks(d, s, &c, &ms)) {
          batch_free(B);
          return rc;
        }
        d.chunks = c;
      }
      btmg_problem* P = nullptr;
      if (int rc = create(&d, &P)) {
        batch_free(B);
        return rc;
      }
      B->probs.push_back(P);
      B->auto_ch.push_back(auto_chunks(d.psi_dtype, d.pg != 0, tiles, nd));
      B->tuned_ms.push_back(ms);
      B->res_off.push_back(off);
      off += 2 * (size_t)P->G;
    }
    B->cyc.assign(n, nullptr);
    B->cyc_psi.assign(n, nullptr);
    B->cycA.assign(n, nullptr);
    B->cycB.assign(n, nullptr);
    if (cudaMallocHost(&B->h_res, sizeof(double) * off) != cudaSuccess ||
        cudaMallocHost(&B->h_err, sizeof(int) * n) != cudaSuccess) {
      batch_free(B);
      return fail(BTMG_ERR_OOM, "batch pinned buffers");
    }
    std::memset(B->h_err, 0, sizeof(int) * n);
    // the persistent coarse launch: one-group problems with FP32 compute and
    // the published correction sweeps, the same sweep count throughout
    B->persist = true;
    B->autotune = autotune != 0;
    for (btmg_problem* P : B->probs)
      if (P->f64 || P->G != 1 || P->d.scat_levels != 0 || P->d.nu_jacobi != B->probs[0]->d.nu_jacobi ||
          !coarse_batch_supported(P->d.nu_jacobi, 32))
        B->persist = false;
    if (B->persist && (cudaMalloc(&B->d_cerr, sizeof(int)) != cudaSuccess ||
                       cudaMallocHost(&B->h_cerr, sizeof(int)) != cudaSuccess)) {
      batch_free(B);
      return fail(BTMG_ERR_OOM, "batch error word");
    }
    if (B->persist) *B->h_cerr = 0;
  } catch (...) {
    batch_free(B);
    return fail(BTMG_ERR_OOM, "host allocation failed");
  }
  *out = B;
  return BTMG_OK;
}

int btmg_destroy_batch(btmg_batch* b) {
  if (b) cudaDeviceSynchronize();
  batch_free(b);
  return BTMG_OK;
}

int btmg_batch_problem(btmg_batch* b, int32_t i, btmg_problem** p) {
  if (!b || !p || i < 0 || i >= (int)b->probs.size()) return fail(BTMG_ERR_INVALID_ARG, "bad batch index");
  *p = b->probs[i];
  return BTMG_OK;
}

int btmg_batch_wait_selftest(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&ws, kCoarseWaitTestBytes) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    if (ws) cudaFree(ws);
    return fail(BTMG_ERR_OOM, "self-test workspace");
  }
  int h = 0;
  cudaError_t e = launch_coarse_wait_selftest(ws, err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(ws);
  cudaFree(err);
  CK(e);
  return h ? fail(BTMG_ERR_TIMEOUT, "bounded wait of the persistent launch gave up (self-test)") : BTMG_OK;
}

int btmg_batch_coarse(const btmg_batch* b, int32_t* persistent, int32_t* tile, int32_t* ctas, double* ms) {
  if (!b) return fail(BTMG_ERR_INVALID_ARG, "null batch");
  if (persistent) *persistent = b->persist ? 1 : 0;
  if (tile) *tile = b->tu;
  if (ctas) *ctas = b->ctas;
  if (ms) *ms = b->coarse_ms;
  return BTMG_OK;
}

int btmg_batch_chunks(const btmg_batch* b, int32_t i, int32_t* chunks, int32_t* auto_chunks_out, double* ms) {
  if (!b || i < 0 || i >= (int)b->probs.size()) return fail(BTMG_ERR_INVALID_ARG, "bad batch index");
  if (chunks) *chunks = b->probs[i]->nchunk;
  if (auto_chunks_out) *auto_chunks_out = b->auto_ch[i];
  if (ms) *ms = b->tuned_ms[i];
  return BTMG_OK;
}

int btmg_solve_batch(btmg_batch* b, void* const* psi, double rtol, int32_t max_cycles, int32_t check_every,
                     btmg_solve_info* infos, void* stream) {
  if (!b || !psi || max_cycles < 1) return fail(BTMG_ERR_INVALID_ARG, "bad batch solve arguments");
  for (size_t i = 0; i < b->probs.size(); ++i)
    if (!psi[i]) return fail(BTMG_ERR_INVALID_ARG, "null psi in batch");
  try {
    return solve_batch(b, psi, rtol, max_cycles, check_every > 0 ? check_every : 1, infos, (cudaStream_t)stream);
  } catch (...) {
    return fail(BTMG_ERR_OOM, "host allocation failed");
  }
}

}  // extern "C"
