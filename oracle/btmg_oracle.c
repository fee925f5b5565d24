/*
 * btmg_oracle.c -- plain, slow, FP64 CPU oracle of the space-angle sawtooth
 * multigrid method for the 2D-space x 2D-angle discretised Boltzmann transport
 * equation (Phillips, Heaney, Chen, Buchan, Pain: "Solving the Discretised
 * Boltzmann Transport Equations using Neural Networks", arXiv 2301.09991).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Every operation is written the way the paper states it: 2D correlations are
 * full (2l+1)x(2l+1) double loops over the printed-form filters, Jacobi sweeps
 * follow Eq. (matrix_full) literally, the cycle follows Fig. (multi_grid_it)
 * step by step.  No blocking, fusion or reordering.  The only parallelism is
 * an OpenMP loop over independent direction planes, which does not change any
 * arithmetic.
 *
 * Readings of points the paper leaves open (each flagged where it is used):
 *   R1  quadrature: collapsed bilinear map of the N_r x N_c rectangular grid
 *       onto each octahedron face, radial projection, patch integrals by
 *       tensor Gauss-Legendre (Sec. 2.2).
 *   R2  direction grid "n_polar x n_azim" = 8 faces of (n_polar/2)x(n_azim/4).
 *   R3  phi = sum_n p_n psi_n with sum p = 4 pi; isotropic scattering source
 *       sigma_s phi / (4 pi); q_n = s per steradian (Sec. 2.2).
 *   R4  residual r = b - A psi per unit area (w_ml -> 1), Eq. (Petrov).
 *   R5  linear ConvFEM filters are derived, not the printed (2x) w_x, w_y.
 *   R6  filters are defined by the operator they discretise (offsets in +x,
 *       +y), not by print orientation.
 *   R7  the printed 1/(dy)^2 prefactor of w_m is dropped (entries sum to 1).
 *   R8  f^{k-Diff} is the literal discretised form of Eqs. (kxx),(kyy),
 *       without the 1/2 of the analytic form (pg_half = 1 restores it).
 *   R9  alpha_r = beta_r = 3 (Sec. 2.6).
 *   R10 halo: psi follows the paper's rule (incoming -> 0, outgoing -> copy
 *       of the adjacent interior node); derived fields (Psi_x, Psi_y, k_x,
 *       k_y) are copied from the nearest interior node; (k psi) halo is
 *       k_halo * psi_halo; corners: incoming in either axis gives 0.
 *   R11 upwind filters as printed in Sec. 2.4 (one-sided, by sign of mu, nu).
 *   R12 coarse equations per unit area and solid angle:
 *       s_{l+1} = sum_children p dx dy s_l / (P dX dY); beta = 1 there.
 *   R13 nu Jacobi sweeps on every level; one PG Jacobi sweep (beta = 3).
 *   R14 no scattering in the coarse / upwind correction operators (the
 *       method as published).  Variant (scat_levels = 1: the levels of the
 *       coarsest angular resolution, N_r = N_c = 1; 2: every level): the
 *       upwind correction sweeps also carry the in-group isotropic
 *       scattering sigma_s phi / (4 pi), each node's directions solved
 *       together with their in-node scattering coupling (node-block
 *       Jacobi, neighbours lagged).  Coarse sigma_s = harmonic sigma_t of
 *       the level times the mean scattering ratio sigma_s / sigma_t of the
 *       present children (S1).
 *   R16 each dimension (nx, ny, N_r, N_c) coarsens to ceil(n/2) until 1;
 *       a missing child counts as 0 in the restriction sum.
 *   R17 harmonic mean of the present children; 0 if any child is 0.
 *   R19 rel = ||r||_W / ||q||_W with W = p_n dx dy (FP64).
 *   R21 N x N nodes, cell centred, dx = L / N.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_MAXLEV 40

/* ------------------------------------------------------------------------ */
/* Public description of a fixed-source problem (Sec. 2.1, Eq. gov-simple). */
typedef struct {
  int32_t nx, ny;          /* nodes in x and y (cell centred)              */
  double lx, ly;           /* domain size                                  */
  int32_t order;           /* ConvFEM polynomial order p: 1, 2 or 3        */
  int32_t n_polar, n_azim; /* direction grid: 8 faces of (n_polar/2)x(n_azim/4) */
  int32_t n_groups;
  const int32_t* region;   /* [ny][nx] region id of each node               */
  int32_t n_regions;
  const double* sigma_t;   /* [n_regions][G] total cross section            */
  const double* sigma_s;   /* [n_regions][G][G] isotropic, [to g][from g']  */
  const double* source;    /* [n_regions][G] isotropic, per steradian       */
  int32_t bc[4];           /* xlo, xhi, ylo, yhi: 0 vacuum, 1 reflective    */
  int32_t pg;              /* 1: PG on the finest level; 0: upwind only     */
  int32_t nu;              /* Jacobi sweeps per level                       */
  double beta_pg;          /* diagonal factor of the fine PG Jacobi (3)     */
  int32_t max_levels;      /* 0: coarsen until every dimension is 1         */
  int32_t pg_half;         /* 1: multiply f^{k-Diff} by 1/2 (analytic form) */
  int32_t ngauss;          /* Gauss points per patch dimension (16)         */
  int32_t scat_levels;     /* R14 variant: 0 off, 1 coarsest angular levels,
                              2 every level                                 */
} or_desc;

typedef struct {
  int nx, ny, nr, nc, nd;
  double dx, dy;
  double *mu, *nu, *xi, *p; /* [nd] */
  double* sigt;             /* [G][ny][nx] */
  double* cratio;           /* [G][ny][nx] in-group sigma_s / sigma_t (S1)  */
} or_level;

typedef struct or_problem {
  or_desc d;
  int G, L, order, l; /* l = filter half width = order */
  double eps_k, a_kabs, a_ksq, a_r;
  /* (2l+1)x(2l+1) filters, w[(v+l)*(2l+1) + (u+l)], u = x offset, v = y offset */
  double wx[49], wy[49], wdxx[49], wdyy[49], wm[49];
  double m1[7], d1[7], s1[7]; /* 1D ConvFEM stencils (dimensionless, h = 1) */
  double* sigs;               /* [G][G][ny][nx] fine, [to][from]            */
  double* src;                /* [G][ny][nx] fine external source           */
  double* extra_q;            /* optional [G][nd][ny][nx] additive source    */
  double *kx_frozen, *ky_frozen; /* optional frozen PG coefficients         */
  or_level lev[OR_MAXLEV];
} or_problem;

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights on [0,1] (Newton on P_n).               */
static void gauss01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-15) {
        /* recompute the derivative at the converged node */
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = pk;
        }
        dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp); /* = 0.5 * 2/((1-z^2) P_n'^2) */
  }
}

int or_gauss01(int n, double* x, double* w) {
  if (n < 1 || n > 256) return -1;
  gauss01(n, x, w);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Octahedral quadrature (Sec. 2.2, Fig. octa).  Face signs (sx, sy, sz);
 * face index f = 4*(sz<0) + 2*(sy<0) + (sx<0).  The face triangle with
 * corners a = sx e_x, b = sy e_y, c = sz e_z carries the rectangular grid
 * (u, t) in [0,1]^2 through X(u,t) = (1-t)((1-u) a + u b) + t c (the edge
 * t = 1 collapses onto c).  Patch (j, i) covers t in [j/nr, (j+1)/nr],
 * u in [i/nc, (i+1)/nc].  On the unit sphere P = X/|X|; the patch area is
 * p = int |dP/du x dP/dt| du dt and the mean direction is int P dS / p.
 * Direction index n = f*nr*nc + j*nc + i.                                 */
static void face_signs(int f, double* sx, double* sy, double* sz) {
  *sx = (f & 1) ? -1.0 : 1.0;
  *sy = (f & 2) ? -1.0 : 1.0;
  *sz = (f & 4) ? -1.0 : 1.0;
}

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Raw (unnormalised) patch integrals for every direction. */
int or_quadrature_raw(int nr, int nc, int ngauss, double* mu, double* nu,
                      double* xi, double* p) {
  if (nr < 1 || nc < 1 || ngauss < 1 || ngauss > 256) return -1;
  double gx[256], gw[256];
  gauss01(ngauss, gx, gw);
  for (int f = 0; f < 8; ++f) {
    double sx, sy, sz;
    face_signs(f, &sx, &sy, &sz);
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < nc; ++i) {
        double A = 0, Mx = 0, My = 0, Mz = 0;
        for (int bt = 0; bt < ngauss; ++bt)
          for (int bu = 0; bu < ngauss; ++bu) {
            double t = (j + gx[bt]) / nr, u = (i + gx[bu]) / nc;
            double w = gw[bt] * gw[bu] / ((double)nr * nc);
            double X[3] = {(1 - t) * (1 - u) * sx, (1 - t) * u * sy, t * sz};
            double Xu[3] = {-(1 - t) * sx, (1 - t) * sy, 0.0};
            double Xt[3] = {-(1 - u) * sx, -u * sy, sz};
            double rr = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
            double P[3] = {X[0] / rr, X[1] / rr, X[2] / rr};
            double pu = P[0] * Xu[0] + P[1] * Xu[1] + P[2] * Xu[2];
            double pt = P[0] * Xt[0] + P[1] * Xt[1] + P[2] * Xt[2];
            double Pu[3], Pt[3], Cr[3];
            for (int k = 0; k < 3; ++k) {
              Pu[k] = (Xu[k] - P[k] * pu) / rr;
              Pt[k] = (Xt[k] - P[k] * pt) / rr;
            }
            cross3(Pu, Pt, Cr);
            double J = sqrt(Cr[0] * Cr[0] + Cr[1] * Cr[1] + Cr[2] * Cr[2]);
            A += w * J;
            Mx += w * J * P[0];
            My += w * J * P[1];
            Mz += w * J * P[2];
          }
        int n = f * nr * nc + j * nc + i;
        p[n] = A;
        mu[n] = Mx / A;
        nu[n] = My / A;
        xi[n] = Mz / A;
      }
  }
  return 0;
}

/* Normalised so that sum_n p_n = 4 pi (Sec. 2.2). */
int or_quadrature(int nr, int nc, int ngauss, double* mu, double* nu, double* xi,
                  double* p) {
  int rc = or_quadrature_raw(nr, nc, ngauss, mu, nu, xi, p);
  if (rc) return rc;
  int nd = 8 * nr * nc;
  double s = 0;
  for (int n = 0; n < nd; ++n) s += p[n];
  for (int n = 0; n < nd; ++n) p[n] *= 4.0 * OR_PI / s;
  return 0;
}

/* Angular coarsening (Sec. 2.5): 2x2 blocks of patches inside a face are
 * merged; the coarse weight is the sum, the coarse direction the
 * weight-averaged mean direction of the union.  A per-face dimension of 1
 * is not merged (R16).                                                     */
static void coarsen_angle(int nr, int nc, const double* mu, const double* nu,
                          const double* xi, const double* p, int nr2, int nc2,
                          double* mu2, double* nu2, double* xi2, double* p2) {
  int fr = (nr > 1) ? 2 : 1, fc = (nc > 1) ? 2 : 1;
  for (int f = 0; f < 8; ++f)
    for (int J = 0; J < nr2; ++J)
      for (int I = 0; I < nc2; ++I) {
        double P = 0, Mx = 0, My = 0, Mz = 0;
        for (int a = 0; a < fr; ++a)
          for (int b = 0; b < fc; ++b) {
            int j = J * fr + a, i = I * fc + b;
            if (j >= nr || i >= nc) continue;
            int n = f * nr * nc + j * nc + i;
            P += p[n];
            Mx += p[n] * mu[n];
            My += p[n] * nu[n];
            Mz += p[n] * xi[n];
          }
        int N = f * nr2 * nc2 + J * nc2 + I;
        p2[N] = P;
        mu2[N] = Mx / P;
        nu2[N] = My / P;
        xi2[N] = Mz / P;
      }
}

/* ------------------------------------------------------------------------ */
/* ConvFEM 1D stencils (Sec. 2.7 and the Appendix).  For polynomial order p
 * the 1D Lagrange element on [0, p] (h = 1) with nodes 0..p has mass
 * M_ab = int N_a N_b, advection C_ab = int N_a N_b' and stiffness
 * K_ab = int N_a' N_b'.  A node of type k (k = 0 is the element corner,
 * shared by two elements; 0 < k < p are interior nodes) has an assembled
 * row of offsets -p..p; ConvFEM averages the rows of the p node types into
 * one stencil valid everywhere, and divides by the lumped mass (the average
 * row sum of the mass, = h).                                               */
static double lagrange(int p, int a, double x) {
  double v = 1.0;
  for (int m = 0; m <= p; ++m)
    if (m != a) v *= (x - m) / (double)(a - m);
  return v;
}

static double lagrange_d(int p, int a, double x) {
  double s = 0.0;
  for (int k = 0; k <= p; ++k) {
    if (k == a) continue;
    double v = 1.0 / (double)(a - k);
    for (int m = 0; m <= p; ++m)
      if (m != a && m != k) v *= (x - m) / (double)(a - m);
    s += v;
  }
  return s;
}

int or_convfem_1d(int p, double* m1, double* d1, double* s1, double* mlumped) {
  if (p < 1 || p > 3) return -1;
  double gx[16], gw[16];
  gauss01(8, gx, gw);
  double M[4][4], C[4][4], K[4][4];
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) {
      double sm = 0, sc = 0, sk = 0;
      for (int q = 0; q < 8; ++q) {
        double x = p * gx[q], w = p * gw[q];
        sm += w * lagrange(p, a, x) * lagrange(p, b, x);
        sc += w * lagrange(p, a, x) * lagrange_d(p, b, x);
        sk += w * lagrange_d(p, a, x) * lagrange_d(p, b, x);
      }
      M[a][b] = sm;
      C[a][b] = sc;
      K[a][b] = sk;
    }
  double am[7] = {0}, ac[7] = {0}, ak[7] = {0};
  for (int k = 0; k < p; ++k) {
    if (k == 0) {
      /* corner: last node of the left element, first node of the right */
      for (int b = 0; b <= p; ++b) {
        am[b - p + p] += M[p][b];
        ac[b - p + p] += C[p][b];
        ak[b - p + p] += K[p][b];
        am[b + p] += M[0][b];
        ac[b + p] += C[0][b];
        ak[b + p] += K[0][b];
      }
    } else {
      for (int b = 0; b <= p; ++b) {
        am[b - k + p] += M[k][b];
        ac[b - k + p] += C[k][b];
        ak[b - k + p] += K[k][b];
      }
    }
  }
  double mL = 0;
  for (int o = 0; o < 2 * p + 1; ++o) mL += am[o] / p;
  for (int o = 0; o < 2 * p + 1; ++o) {
    m1[o] = am[o] / p / mL;
    d1[o] = ac[o] / p / mL;
    s1[o] = ak[o] / p / mL;
  }
  if (mlumped) *mlumped = mL;
  return 0;
}

/* 2D filters as tensor products of the averaged 1D stencils (the 2D node
 * types are products of the 1D ones, so the 2D average is the product of
 * the 1D averages), in physical units for spacings dx, dy.  Layout
 * w[(v+l)*(2l+1) + (u+l)] with u the x offset and v the y offset (R6).     */
int or_filters_2d(int p, double dx, double dy, double* wx, double* wy,
                  double* wdxx, double* wdyy, double* wm) {
  double m1[7], d1[7], s1[7];
  int rc = or_convfem_1d(p, m1, d1, s1, NULL);
  if (rc) return rc;
  int w = 2 * p + 1;
  for (int v = 0; v < w; ++v)
    for (int u = 0; u < w; ++u) {
      wx[v * w + u] = d1[u] * m1[v] / dx;
      wy[v * w + u] = m1[u] * d1[v] / dy;
      wdxx[v * w + u] = s1[u] * m1[v] / (dx * dx);
      wdyy[v * w + u] = m1[u] * s1[v] / (dy * dy);
      wm[v * w + u] = m1[u] * m1[v];
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Problem set-up: materials per node (R21), level hierarchy (Sec. 2.5).    */
static int ceil_half(int n) { return (n > 1) ? (n + 1) / 2 : 1; }

void or_destroy(or_problem* P) {
  if (!P) return;
  for (int l = 0; l < P->L; ++l) {
    free(P->lev[l].mu);
    free(P->lev[l].nu);
    free(P->lev[l].xi);
    free(P->lev[l].p);
    free(P->lev[l].sigt);
    free(P->lev[l].cratio);
  }
  free(P->sigs);
  free(P->src);
  free(P->extra_q);
  free(P->kx_frozen);
  free(P->ky_frozen);
  free(P);
}

or_problem* or_create(const or_desc* d) {
  if (!d || d->nx < 1 || d->ny < 1 || d->n_groups < 1 || d->n_regions < 1)
    return NULL;
  if (d->n_polar < 2 || d->n_azim < 4 || d->n_polar % 2 || d->n_azim % 4)
    return NULL;
  if (d->order < 1 || d->order > 3 || d->nu < 0) return NULL;
  if (d->scat_levels < 0 || d->scat_levels > 2) return NULL;
  or_problem* P = (or_problem*)calloc(1, sizeof(or_problem));
  if (!P) return NULL;
  P->d = *d;
  P->d.region = NULL;
  P->d.sigma_t = P->d.sigma_s = P->d.source = NULL;
  if (P->d.ngauss <= 0) P->d.ngauss = 16;
  if (P->d.beta_pg <= 0) P->d.beta_pg = 3.0;
  const int G = d->n_groups, nx = d->nx, ny = d->ny;
  P->G = G;
  P->order = d->order;
  P->l = d->order;
  /* Sec. 2.6: eps_k = 0.001, alpha_kabs = 2^p/16, alpha_ksquare = 2^p/2;
   * alpha_r = beta_r = 3 (R9). */
  P->eps_k = 1e-3;
  P->a_kabs = pow(2.0, d->order) / 16.0;
  P->a_ksq = pow(2.0, d->order) / 2.0;
  P->a_r = 3.0;
  double dx = d->lx / nx, dy = d->ly / ny, mL;
  or_convfem_1d(d->order, P->m1, P->d1, P->s1, &mL);
  or_filters_2d(d->order, dx, dy, P->wx, P->wy, P->wdxx, P->wdyy, P->wm);

  P->sigs = (double*)calloc((size_t)G * G * nx * ny, sizeof(double));
  P->src = (double*)calloc((size_t)G * nx * ny, sizeof(double));
  or_level* L0 = &P->lev[0];
  L0->sigt = (double*)calloc((size_t)G * nx * ny, sizeof(double));
  L0->cratio = (double*)calloc((size_t)G * nx * ny, sizeof(double));
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int rg = d->region[y * nx + x];
      if (rg < 0 || rg >= d->n_regions) {
        or_destroy(P);
        return NULL;
      }
      for (int g = 0; g < G; ++g) {
        L0->sigt[((size_t)g * ny + y) * nx + x] = d->sigma_t[rg * G + g];
        if (d->sigma_t[rg * G + g] > 0.0)
          L0->cratio[((size_t)g * ny + y) * nx + x] =
              d->sigma_s[(rg * G + g) * G + g] / d->sigma_t[rg * G + g];
        P->src[((size_t)g * ny + y) * nx + x] = d->source[rg * G + g];
        for (int h = 0; h < G; ++h)
          P->sigs[(((size_t)g * G + h) * ny + y) * nx + x] =
              d->sigma_s[(rg * G + g) * G + h];
      }
    }
  L0->nx = nx;
  L0->ny = ny;
  L0->nr = d->n_polar / 2;
  L0->nc = d->n_azim / 4;
  L0->nd = 8 * L0->nr * L0->nc;
  L0->dx = dx;
  L0->dy = dy;
  L0->mu = (double*)malloc(sizeof(double) * L0->nd);
  L0->nu = (double*)malloc(sizeof(double) * L0->nd);
  L0->xi = (double*)malloc(sizeof(double) * L0->nd);
  L0->p = (double*)malloc(sizeof(double) * L0->nd);
  or_quadrature(L0->nr, L0->nc, P->d.ngauss, L0->mu, L0->nu, L0->xi, L0->p);
  P->L = 1;
  while (P->L < OR_MAXLEV) {
    or_level* A = &P->lev[P->L - 1];
    if (d->max_levels > 0 && P->L >= d->max_levels) break;
    if (A->nx == 1 && A->ny == 1 && A->nr == 1 && A->nc == 1) break;
    or_level* B = &P->lev[P->L];
    B->nx = ceil_half(A->nx);
    B->ny = ceil_half(A->ny);
    B->nr = ceil_half(A->nr);
    B->nc = ceil_half(A->nc);
    B->nd = 8 * B->nr * B->nc;
    B->dx = (A->nx > 1) ? 2.0 * A->dx : A->dx;
    B->dy = (A->ny > 1) ? 2.0 * A->dy : A->dy;
    B->mu = (double*)malloc(sizeof(double) * B->nd);
    B->nu = (double*)malloc(sizeof(double) * B->nd);
    B->xi = (double*)malloc(sizeof(double) * B->nd);
    B->p = (double*)malloc(sizeof(double) * B->nd);
    coarsen_angle(A->nr, A->nc, A->mu, A->nu, A->xi, A->p, B->nr, B->nc, B->mu,
                  B->nu, B->xi, B->p);
    /* harmonic average of the present spatial children (R17) */
    B->sigt = (double*)calloc((size_t)G * B->nx * B->ny, sizeof(double));
    B->cratio = (double*)calloc((size_t)G * B->nx * B->ny, sizeof(double));
    int fx = (A->nx > 1) ? 2 : 1, fy = (A->ny > 1) ? 2 : 1;
    for (int g = 0; g < G; ++g)
      for (int Y = 0; Y < B->ny; ++Y)
        for (int X = 0; X < B->nx; ++X) {
          int cnt = 0, zero = 0;
          double inv = 0, cr = 0;
          for (int b = 0; b < fy; ++b)
            for (int a = 0; a < fx; ++a) {
              int x = X * fx + a, y = Y * fy + b;
              if (x >= A->nx || y >= A->ny) continue;
              double s = A->sigt[((size_t)g * A->ny + y) * A->nx + x];
              ++cnt;
              cr += A->cratio[((size_t)g * A->ny + y) * A->nx + x];
              if (s == 0.0) zero = 1;
              else inv += 1.0 / s;
            }
          B->sigt[((size_t)g * B->ny + Y) * B->nx + X] = zero ? 0.0 : cnt / inv;
          B->cratio[((size_t)g * B->ny + Y) * B->nx + X] = cr / cnt; /* S1 */
        }
    P->L++;
  }
  return P;
}

int or_num_levels(const or_problem* P) { return P->L; }

int or_level_dims(const or_problem* P, int l, int32_t* dims /*nx,ny,nr,nc,nd*/,
                  double* dxdy) {
  if (l < 0 || l >= P->L) return -1;
  const or_level* A = &P->lev[l];
  dims[0] = A->nx;
  dims[1] = A->ny;
  dims[2] = A->nr;
  dims[3] = A->nc;
  dims[4] = A->nd;
  if (dxdy) {
    dxdy[0] = A->dx;
    dxdy[1] = A->dy;
  }
  return 0;
}

int or_level_quad(const or_problem* P, int l, double* mu, double* nu, double* xi,
                  double* p) {
  if (l < 0 || l >= P->L) return -1;
  const or_level* A = &P->lev[l];
  memcpy(mu, A->mu, sizeof(double) * A->nd);
  memcpy(nu, A->nu, sizeof(double) * A->nd);
  memcpy(xi, A->xi, sizeof(double) * A->nd);
  memcpy(p, A->p, sizeof(double) * A->nd);
  return 0;
}

int or_level_sigt(const or_problem* P, int l, double* out) {
  if (l < 0 || l >= P->L) return -1;
  const or_level* A = &P->lev[l];
  memcpy(out, A->sigt, sizeof(double) * P->G * A->nx * A->ny);
  return 0;
}
/* In-group scattering ratio per node of level l (S1), [G][ny][nx]. */
int or_level_cratio(const or_problem* P, int l, double* out) {
  if (l < 0 || l >= P->L) return -1;
  const or_level* A = &P->lev[l];
  memcpy(out, A->cratio, sizeof(double) * P->G * A->nx * A->ny);
  return 0;
}

int or_get_filters(const or_problem* P, double* wx, double* wy, double* wdxx,
                   double* wdyy, double* wm) {
  int w = 2 * P->l + 1;
  memcpy(wx, P->wx, sizeof(double) * w * w);
  memcpy(wy, P->wy, sizeof(double) * w * w);
  memcpy(wdxx, P->wdxx, sizeof(double) * w * w);
  memcpy(wdyy, P->wdyy, sizeof(double) * w * w);
  memcpy(wm, P->wm, sizeof(double) * w * w);
  return 0;
}

/* Optional additive anisotropic source [G][nd][ny][nx] (manufactured
 * solutions); NULL removes it. */
int or_set_extra_source(or_problem* P, const double* q) {
  size_t n = (size_t)P->G * P->lev[0].nd * P->lev[0].nx * P->lev[0].ny;
  free(P->extra_q);
  P->extra_q = NULL;
  if (!q) return 0;
  P->extra_q = (double*)malloc(sizeof(double) * n);
  memcpy(P->extra_q, q, sizeof(double) * n);
  return 0;
}

/* Freeze k_x, k_y ([G][nd][ny][nx]) for every PG evaluation; NULL unfreezes. */
int or_set_frozen_k(or_problem* P, const double* kx, const double* ky) {
  size_t n = (size_t)P->G * P->lev[0].nd * P->lev[0].nx * P->lev[0].ny;
  free(P->kx_frozen);
  free(P->ky_frozen);
  P->kx_frozen = P->ky_frozen = NULL;
  if (!kx || !ky) return 0;
  P->kx_frozen = (double*)malloc(sizeof(double) * n);
  P->ky_frozen = (double*)malloc(sizeof(double) * n);
  memcpy(P->kx_frozen, kx, sizeof(double) * n);
  memcpy(P->ky_frozen, ky, sizeof(double) * n);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Halo rule (Sec. 2.3, R10).  sx, sy are the signs of mu, nu.              */
static double halo_val(const double* f, int nx, int ny, int x, int y, double sx,
                       double sy, const int32_t* bc, int derived) {
  if (!derived) {
    if (x < 0 && bc[0] == 0 && sx > 0) return 0.0;
    if (x >= nx && bc[1] == 0 && sx < 0) return 0.0;
    if (y < 0 && bc[2] == 0 && sy > 0) return 0.0;
    if (y >= ny && bc[3] == 0 && sy < 0) return 0.0;
  }
  int cx = x < 0 ? 0 : (x >= nx ? nx - 1 : x);
  int cy = y < 0 ? 0 : (y >= ny ? ny - 1 : y);
  return f[(size_t)cy * nx + cx];
}

/* Plain 2D correlation f(a; w)|_{x,y} = sum_{u,v} w_{u,v} a_ext(x+u, y+v). */
static double corr(const double* w, int l, const double* a, int nx, int ny, int x,
                   int y, double sx, double sy, const int32_t* bc, int derived) {
  double s = 0.0;
  int W = 2 * l + 1;
  for (int v = -l; v <= l; ++v)
    for (int u = -l; u <= l; ++u)
      s += w[(v + l) * W + (u + l)] *
           halo_val(a, nx, ny, x + u, y + v, sx, sy, bc, derived);
  return s;
}

/* Correlation of the product k_ext * psi_ext (R10). */
static double corr_prod(const double* w, int l, const double* k, const double* a,
                        int nx, int ny, int x, int y, double sx, double sy,
                        const int32_t* bc) {
  double s = 0.0;
  int W = 2 * l + 1;
  for (int v = -l; v <= l; ++v)
    for (int u = -l; u <= l; ++u)
      s += w[(v + l) * W + (u + l)] *
           halo_val(k, nx, ny, x + u, y + v, sx, sy, bc, 1) *
           halo_val(a, nx, ny, x + u, y + v, sx, sy, bc, 0);
  return s;
}

/* Anisotropic PG coefficients (Sec. 2.6, Eq. ano-k) for one direction plane:
 *   Psi_x = f(Psi; w_x),  R_x = alpha_r mu f(Psi_x; w_m - I),
 *   k_x = min{ dx|mu|, a_kabs |R_x| dx / (eps + |Psi_x|),
 *              a_ksq R_x^2 dx / (eps + |mu| Psi_x^2) }   (y likewise).     */
static void pg_kfields(const or_problem* P, int n, const double* psi, double* Px,
                       double* Py, double* kx, double* ky) {
  const or_level* A = &P->lev[0];
  const int nx = A->nx, ny = A->ny, l = P->l, W = 2 * l + 1;
  const double mu = A->mu[n], nu = A->nu[n];
  const double sx = mu > 0 ? 1.0 : -1.0, sy = nu > 0 ? 1.0 : -1.0;
  const int32_t* bc = P->d.bc;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      Px[y * nx + x] = corr(P->wx, l, psi, nx, ny, x, y, sx, sy, bc, 0);
      Py[y * nx + x] = corr(P->wy, l, psi, nx, ny, x, y, sx, sy, bc, 0);
    }
  double wmI[49];
  memcpy(wmI, P->wm, sizeof(double) * W * W);
  wmI[l * W + l] -= 1.0; /* m_L^{-1} m - I */
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      double Rx = P->a_r * mu * corr(wmI, l, Px, nx, ny, x, y, sx, sy, bc, 1);
      double Ry = P->a_r * nu * corr(wmI, l, Py, nx, ny, x, y, sx, sy, bc, 1);
      double kxmax = A->dx * fabs(mu), kymax = A->dy * fabs(nu);
      double kxabs = P->a_kabs * fabs(Rx) * A->dx / (P->eps_k + fabs(Px[i]));
      double kyabs = P->a_kabs * fabs(Ry) * A->dy / (P->eps_k + fabs(Py[i]));
      double kxsq = P->a_ksq * Rx * Rx * A->dx / (P->eps_k + fabs(mu) * Px[i] * Px[i]);
      double kysq = P->a_ksq * Ry * Ry * A->dy / (P->eps_k + fabs(nu) * Py[i] * Py[i]);
      double a = kxmax < kxabs ? kxmax : kxabs;
      kx[i] = a < kxsq ? a : kxsq;
      double b = kymax < kyabs ? kymax : kyabs;
      ky[i] = b < kysq ? b : kysq;
    }
}

/* Fine operator for one (g, n) plane: r = b_n - A psi_n (R4).  b is the
 * isotropic part [ny][nx]; extra (nullable) an additive per-direction part.
 * With pg = 1 (Eq. Petrov):
 *   A psi = mu Psi_x + nu Psi_y + f^{kDiff}(psi; k_x, w_Dxx)
 *           + f^{kDiff}(psi; k_y, w_Dyy) + sigma_t psi,
 *   f^{kDiff}(psi; k, w) = f(k psi; w) + k f(psi; w) - psi f(k; w)   (Eq. kxx).
 * With pg = 0 the upwind operator of level 0 (Sec. 2.3/2.4).              */
static void upwind_apply_plane(const or_problem* P, int lev, int g, int n,
                               const double* a, double* out);

static void fine_residual_plane(const or_problem* P, int g, int n, const double* psi,
                                const double* b, const double* extra, double* r,
                                const double* kx_in, const double* ky_in,
                                double* kx_out, double* ky_out) {
  const or_level* A = &P->lev[0];
  const int nx = A->nx, ny = A->ny, l = P->l;
  const size_t np = (size_t)nx * ny;
  const double mu = A->mu[n], nu = A->nu[n];
  const double sx = mu > 0 ? 1.0 : -1.0, sy = nu > 0 ? 1.0 : -1.0;
  const int32_t* bc = P->d.bc;
  const double* sigt = A->sigt + (size_t)g * np;
  if (!P->d.pg) {
    double* Ap = (double*)malloc(sizeof(double) * np);
    upwind_apply_plane(P, 0, g, n, psi, Ap);
    for (size_t i = 0; i < np; ++i) r[i] = b[i] + (extra ? extra[i] : 0.0) - Ap[i];
    free(Ap);
    return;
  }
  double* Px = (double*)malloc(sizeof(double) * np);
  double* Py = (double*)malloc(sizeof(double) * np);
  double* kx = (double*)malloc(sizeof(double) * np);
  double* ky = (double*)malloc(sizeof(double) * np);
  pg_kfields(P, n, psi, Px, Py, kx, ky);
  if (kx_in) memcpy(kx, kx_in, sizeof(double) * np);
  if (ky_in) memcpy(ky, ky_in, sizeof(double) * np);
  if (kx_out) memcpy(kx_out, kx, sizeof(double) * np);
  if (ky_out) memcpy(ky_out, ky, sizeof(double) * np);
  const double half = P->d.pg_half ? 0.5 : 1.0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      double Dx = corr_prod(P->wdxx, l, kx, psi, nx, ny, x, y, sx, sy, bc) +
                  kx[i] * corr(P->wdxx, l, psi, nx, ny, x, y, sx, sy, bc, 0) -
                  psi[i] * corr(P->wdxx, l, kx, nx, ny, x, y, sx, sy, bc, 1);
      double Dy = corr_prod(P->wdyy, l, ky, psi, nx, ny, x, y, sx, sy, bc) +
                  ky[i] * corr(P->wdyy, l, psi, nx, ny, x, y, sx, sy, bc, 0) -
                  psi[i] * corr(P->wdyy, l, ky, nx, ny, x, y, sx, sy, bc, 1);
      double Apsi = mu * Px[i] + nu * Py[i] + half * (Dx + Dy) + sigt[i] * psi[i];
      r[i] = b[i] + (extra ? extra[i] : 0.0) - Apsi;
    }
  free(Px);
  free(Py);
  free(kx);
  free(ky);
}

/* Upwind operator of level lev (Sec. 2.3, filters of Sec. 2.4, R11):
 *   mu>0: mu (a(x) - a(x-1))/dX,  mu<0: mu (a(x+1) - a(x))/dX,  y likewise,
 *   plus sigma_t a.  Halo values by the paper's rule.                      */
static void upwind_apply_plane(const or_problem* P, int lev, int g, int n,
                               const double* a, double* out) {
  const or_level* A = &P->lev[lev];
  const int nx = A->nx, ny = A->ny;
  const double mu = A->mu[n], nu = A->nu[n];
  const double sx = mu > 0 ? 1.0 : -1.0, sy = nu > 0 ? 1.0 : -1.0;
  const int32_t* bc = P->d.bc;
  const double* sigt = A->sigt + (size_t)g * nx * ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double c = a[(size_t)y * nx + x];
      double ax = (mu > 0) ? (c - halo_val(a, nx, ny, x - 1, y, sx, sy, bc, 0)) / A->dx
                           : (halo_val(a, nx, ny, x + 1, y, sx, sy, bc, 0) - c) / A->dx;
      double ay = (nu > 0) ? (c - halo_val(a, nx, ny, x, y - 1, sx, sy, bc, 0)) / A->dy
                           : (halo_val(a, nx, ny, x, y + 1, sx, sy, bc, 0) - c) / A->dy;
      out[(size_t)y * nx + x] = mu * ax + nu * ay + sigt[(size_t)y * nx + x] * c;
    }
}

/* Upwind diagonal d = |mu|/dX + |nu|/dY + sigma_t (Eq. matrix_full, beta=1). */
static double upwind_diag(const or_level* A, int g, int n, int x, int y) {
  return fabs(A->mu[n]) / A->dx + fabs(A->nu[n]) / A->dy +
         A->sigt[((size_t)g * A->ny + y) * A->nx + x];
}

/* ------------------------------------------------------------------------ */
/* Scalar flux phi_g = sum_n p_n psi_{n,g} (Sec. 2.2).                       */
int or_scalar_flux(const or_problem* P, const double* psi, double* phi) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny;
  for (int g = 0; g < P->G; ++g) {
    double* f = phi + (size_t)g * np;
    for (size_t i = 0; i < np; ++i) f[i] = 0.0;
    for (int n = 0; n < A->nd; ++n) {
      const double* s = psi + ((size_t)g * A->nd + n) * np;
      for (size_t i = 0; i < np; ++i) f[i] += A->p[n] * s[i];
    }
  }
  return 0;
}

/* Isotropic right-hand side of group g:
 *   b_g = s_g + sum_{g'} sigma_s[g <- g'] phi_g' / (4 pi)     (R3).        */
static void group_rhs(const or_problem* P, int g, const double* phi, double* b) {
  const size_t np = (size_t)P->lev[0].nx * P->lev[0].ny;
  for (size_t i = 0; i < np; ++i) {
    double v = P->src[(size_t)g * np + i];
    for (int h = 0; h < P->G; ++h)
      v += P->sigs[((size_t)g * P->G + h) * np + i] * phi[(size_t)h * np + i] /
           (4.0 * OR_PI);
    b[i] = v;
  }
}

/* Same, but with the in-group term taken from phi_self and the other groups
 * from phi (block Gauss-Seidel over groups). */
static void group_rhs_fixed(const or_problem* P, int g, const double* phi, double* q) {
  const size_t np = (size_t)P->lev[0].nx * P->lev[0].ny;
  for (size_t i = 0; i < np; ++i) {
    double v = P->src[(size_t)g * np + i];
    for (int h = 0; h < P->G; ++h)
      if (h != g)
        v += P->sigs[((size_t)g * P->G + h) * np + i] * phi[(size_t)h * np + i] /
             (4.0 * OR_PI);
    q[i] = v;
  }
}

/* Residual of one group given the fixed (other-group) source q and the
 * group's own angular flux: r = q + sigma_s[g<-g] phi_g/(4 pi) - A psi_g.
 * Also returns the weighted norms ||r||_W^2 and ||q||_W^2 (R19).          */
static void group_residual(const or_problem* P, int g, const double* psi_g,
                           const double* q, double* r, double* rn2, double* qn2) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny;
  double* phi = (double*)calloc(np, sizeof(double));
  double* b = (double*)malloc(sizeof(double) * np);
  for (int n = 0; n < A->nd; ++n)
    for (size_t i = 0; i < np; ++i) phi[i] += A->p[n] * psi_g[(size_t)n * np + i];
  const double* sgg = P->sigs + ((size_t)g * P->G + g) * np;
  for (size_t i = 0; i < np; ++i) b[i] = q[i] + sgg[i] * phi[i] / (4.0 * OR_PI);
#pragma omp parallel for schedule(dynamic)
  for (int n = 0; n < A->nd; ++n) {
    size_t off = (size_t)n * np, goff = ((size_t)g * A->nd + n) * np;
    fine_residual_plane(P, g, n, psi_g + off, b, P->extra_q ? P->extra_q + goff : NULL,
                        r + off, P->kx_frozen ? P->kx_frozen + goff : NULL,
                        P->ky_frozen ? P->ky_frozen + goff : NULL, NULL, NULL);
  }
  double sr = 0, sq = 0;
  for (int n = 0; n < A->nd; ++n)
    for (size_t i = 0; i < np; ++i) {
      double v = r[(size_t)n * np + i];
      sr += A->p[n] * A->dx * A->dy * v * v;
      double e = q[i] + (P->extra_q ? P->extra_q[((size_t)g * A->nd + n) * np + i] : 0.0);
      sq += A->p[n] * A->dx * A->dy * e * e;
    }
  *rn2 = sr;
  *qn2 = sq;
  free(phi);
  free(b);
}

/* r = b - A psi for every group, with b from the current phi of all groups. */
int or_apply(const or_problem* P, const double* psi, double* r) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny;
  double* phi = (double*)malloc(sizeof(double) * np * P->G);
  double* b = (double*)malloc(sizeof(double) * np);
  or_scalar_flux(P, psi, phi);
  for (int g = 0; g < P->G; ++g) {
    group_rhs(P, g, phi, b);
#pragma omp parallel for schedule(dynamic)
    for (int n = 0; n < A->nd; ++n) {
      size_t off = ((size_t)g * A->nd + n) * np;
      fine_residual_plane(P, g, n, psi + off, b, P->extra_q ? P->extra_q + off : NULL,
                          r + off, P->kx_frozen ? P->kx_frozen + off : NULL,
                          P->ky_frozen ? P->ky_frozen + off : NULL, NULL, NULL);
    }
  }
  free(phi);
  free(b);
  return 0;
}

/* r = b - A psi for a sample of (group, direction) planes only: out holds
 * nsel planes [nsel][ny][nx], plane s is (g, n) = (sel[2s], sel[2s+1]).
 * b still uses the scalar flux of all directions.  Same arithmetic as
 * or_apply, restricted to the requested planes (large-problem checks).   */
int or_apply_planes(const or_problem* P, const double* psi, const int32_t* sel, int nsel,
                    double* out) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny;
  double* phi = (double*)malloc(sizeof(double) * np * P->G);
  double* b = (double*)malloc(sizeof(double) * np * P->G);
  or_scalar_flux(P, psi, phi);
  for (int g = 0; g < P->G; ++g) group_rhs(P, g, phi, b + (size_t)g * np);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < nsel; ++s) {
    int g = sel[2 * s], n = sel[2 * s + 1];
    size_t off = ((size_t)g * A->nd + n) * np;
    fine_residual_plane(P, g, n, psi + off, b + (size_t)g * np,
                        P->extra_q ? P->extra_q + off : NULL, out + (size_t)s * np,
                        P->kx_frozen ? P->kx_frozen + off : NULL,
                        P->ky_frozen ? P->ky_frozen + off : NULL, NULL, NULL);
  }
  free(phi);
  free(b);
  return 0;
}

/* PG coefficients of every plane (for tests and for freezing k). */
int or_kfields(const or_problem* P, const double* psi, double* kx, double* ky) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny;
#pragma omp parallel for schedule(dynamic)
  for (int gn = 0; gn < P->G * A->nd; ++gn) {
    int n = gn % A->nd;
    size_t off = (size_t)gn * np;
    double* Px = (double*)malloc(sizeof(double) * np);
    double* Py = (double*)malloc(sizeof(double) * np);
    pg_kfields(P, n, psi + off, Px, Py, kx + off, ky + off);
    free(Px);
    free(Py);
  }
  return 0;
}

/* Upwind operator of any level applied to a full level-sized field
 * ([G][nd][ny][nx]); exposed for tests. */
int or_upwind_apply(const or_problem* P, int lev, const double* a, double* out) {
  if (lev < 0 || lev >= P->L) return -1;
  const or_level* A = &P->lev[lev];
  const size_t np = (size_t)A->nx * A->ny;
  for (int g = 0; g < P->G; ++g)
    for (int n = 0; n < A->nd; ++n) {
      size_t off = ((size_t)g * A->nd + n) * np;
      upwind_apply_plane(P, lev, g, n, a + off, out + off);
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One Jacobi sweep of the upwind system A_up delta = s on level lev, group g
 * (Eq. matrix_full with beta = 1):  delta <- delta + d^{-1} (s - A_up delta).
 * Simultaneous update: every point uses the old iterate.                   */
static void jacobi_upwind_group(const or_problem* P, int lev, int g, const double* s,
                                double* delta, int sweeps) {
  const or_level* A = &P->lev[lev];
  const size_t np = (size_t)A->nx * A->ny;
#pragma omp parallel for schedule(dynamic)
  for (int n = 0; n < A->nd; ++n) {
    double* Ad = (double*)malloc(sizeof(double) * np);
    double* d = delta + (size_t)n * np;
    const double* sn = s + (size_t)n * np;
    for (int k = 0; k < sweeps; ++k) {
      upwind_apply_plane(P, lev, g, n, d, Ad);
      for (int y = 0; y < A->ny; ++y)
        for (int x = 0; x < A->nx; ++x) {
          size_t i = (size_t)y * A->nx + x;
          d[i] += (sn[i] - Ad[i]) / upwind_diag(A, g, n, x, y);
        }
    }
    free(Ad);
  }
}

/* Does level lev carry the in-group scattering in its upwind sweeps (R14
 * variant)?                                                               */
static int scat_on(const or_problem* P, int lev) {
  if (P->d.scat_levels == 2) return 1;
  if (P->d.scat_levels == 1) return P->lev[lev].nr == 1 && P->lev[lev].nc == 1;
  return 0;
}

/* One node-block Jacobi sweep with the in-node scattering (R14 variant).
 * With the neighbours taken from the old iterate, the directions of one node
 * solve together
 *   d_n delta_n - kappa sum_m p_m delta_m = s_n + d_n delta_n^old - (A_up delta^old)_n,
 * kappa = sigma_s / (4 pi) (R3, S1).  Dividing by d_n, the right-hand side
 * is the plain Jacobi update a_n; the system is the identity plus a rank-one
 * term, so with Phi = sum_m p_m delta_m:
 *   delta_n = a_n + kappa Phi / d_n,   Phi = (sum_n p_n a_n) / (1 - kappa sum_n p_n / d_n). */
static void jacobi_scat_group(const or_problem* P, int lev, int g, const double* s,
                              double* delta, int sweeps) {
  const or_level* A = &P->lev[lev];
  const size_t np = (size_t)A->nx * A->ny;
  double* a = (double*)malloc(sizeof(double) * np * A->nd);
  for (int k = 0; k < sweeps; ++k) {
#pragma omp parallel for schedule(dynamic)
    for (int n = 0; n < A->nd; ++n) {
      double* an = a + (size_t)n * np;
      const double* d = delta + (size_t)n * np;
      const double* sn = s + (size_t)n * np;
      upwind_apply_plane(P, lev, g, n, d, an);
      for (int y = 0; y < A->ny; ++y)
        for (int x = 0; x < A->nx; ++x) {
          size_t i = (size_t)y * A->nx + x;
          an[i] = d[i] + (sn[i] - an[i]) / upwind_diag(A, g, n, x, y);
        }
    }
#pragma omp parallel for
    for (int y = 0; y < A->ny; ++y)
      for (int x = 0; x < A->nx; ++x) {
        size_t i = (size_t)y * A->nx + x, gi = (size_t)g * np + i;
        double kappa = A->cratio[gi] * A->sigt[gi] / (4.0 * OR_PI);
        double spa = 0.0, spd = 0.0;
        for (int n = 0; n < A->nd; ++n) {
          spa += A->p[n] * a[(size_t)n * np + i];
          spd += A->p[n] / upwind_diag(A, g, n, x, y);
        }
        double Phi = spa / (1.0 - kappa * spd);
        for (int n = 0; n < A->nd; ++n)
          delta[(size_t)n * np + i] = a[(size_t)n * np + i] + kappa * Phi / upwind_diag(A, g, n, x, y);
      }
  }
  free(a);
}

/* Restriction level lev -> lev+1 for one group's correction source
 * (Sec. 2.5, R12, R16): s_C = sum_children p_c dx dy s_c / (P_C dX dY).
 * Children: 2 (or 1) in each of x, y, polar and azimuth; missing -> 0.     */
static void restrict_group(const or_problem* P, int lev, const double* s, double* S) {
  const or_level* A = &P->lev[lev];
  const or_level* B = &P->lev[lev + 1];
  const int fx = (A->nx > 1) ? 2 : 1, fy = (A->ny > 1) ? 2 : 1;
  const int fr = (A->nr > 1) ? 2 : 1, fc = (A->nc > 1) ? 2 : 1;
  for (int f = 0; f < 8; ++f)
    for (int J = 0; J < B->nr; ++J)
      for (int I = 0; I < B->nc; ++I) {
        int N = f * B->nr * B->nc + J * B->nc + I;
        for (int Y = 0; Y < B->ny; ++Y)
          for (int X = 0; X < B->nx; ++X) {
            double acc = 0.0;
            for (int a = 0; a < fr; ++a)
              for (int c = 0; c < fc; ++c) {
                int j = J * fr + a, i = I * fc + c;
                if (j >= A->nr || i >= A->nc) continue;
                int n = f * A->nr * A->nc + j * A->nc + i;
                for (int yy = 0; yy < fy; ++yy)
                  for (int xx = 0; xx < fx; ++xx) {
                    int x = X * fx + xx, y = Y * fy + yy;
                    if (x >= A->nx || y >= A->ny) continue;
                    acc += A->p[n] * A->dx * A->dy *
                           s[((size_t)n * A->ny + y) * A->nx + x];
                  }
              }
            S[((size_t)N * B->ny + Y) * B->nx + X] = acc / (B->p[N] * B->dx * B->dy);
          }
      }
}

/* UpSamp (Sec. 2.5): every fine unknown takes the value of its coarse parent. */
static void prolong_group(const or_problem* P, int lev, const double* D, double* d) {
  const or_level* A = &P->lev[lev];
  const or_level* B = &P->lev[lev + 1];
  const int fx = (A->nx > 1) ? 2 : 1, fy = (A->ny > 1) ? 2 : 1;
  const int fr = (A->nr > 1) ? 2 : 1, fc = (A->nc > 1) ? 2 : 1;
  for (int f = 0; f < 8; ++f)
    for (int j = 0; j < A->nr; ++j)
      for (int i = 0; i < A->nc; ++i) {
        int n = f * A->nr * A->nc + j * A->nc + i;
        int N = f * B->nr * B->nc + (j / fr) * B->nc + (i / fc);
        for (int y = 0; y < A->ny; ++y)
          for (int x = 0; x < A->nx; ++x)
            d[((size_t)n * A->ny + y) * A->nx + x] =
                D[((size_t)N * B->ny + y / fy) * B->nx + x / fx];
      }
}

static size_t level_size(const or_problem* P, int l) {
  return (size_t)P->lev[l].nd * P->lev[l].nx * P->lev[l].ny;
}

/* Exposed single steps (one group, level-shaped buffers [nd][ny][nx]). */
int or_restrict(const or_problem* P, int lev, const double* fine, double* coarse) {
  if (lev < 0 || lev + 1 >= P->L) return -1;
  restrict_group(P, lev, fine, coarse);
  return 0;
}
int or_prolong(const or_problem* P, int lev, const double* coarse, double* fine) {
  if (lev < 0 || lev + 1 >= P->L) return -1;
  prolong_group(P, lev, coarse, fine);
  return 0;
}
int or_jacobi_upwind(const or_problem* P, int lev, int g, const double* s,
                     double* delta, int sweeps) {
  if (lev < 0 || lev >= P->L || g < 0 || g >= P->G) return -1;
  if (scat_on(P, lev))
    jacobi_scat_group(P, lev, g, s, delta, sweeps);
  else
    jacobi_upwind_group(P, lev, g, s, delta, sweeps);
  return 0;
}

/* Fine PG Jacobi for one group (Eq. matrix_full, beta = beta_pg; with pg = 0
 * the upwind residual and beta = 1):
 *   psi <- psi + (beta d)^{-1} (b - A psi).                                */
static void pg_jacobi_group(const or_problem* P, int g, double* psi_g, const double* q,
                            int sweeps) {
  const or_level* A = &P->lev[0];
  const size_t n1 = level_size(P, 0), np = (size_t)A->nx * A->ny;
  double* r = (double*)malloc(sizeof(double) * n1);
  const double beta = P->d.pg ? P->d.beta_pg : 1.0;
  for (int k = 0; k < sweeps; ++k) {
    double rn, qn;
    group_residual(P, g, psi_g, q, r, &rn, &qn);
    for (int n = 0; n < A->nd; ++n)
      for (int y = 0; y < A->ny; ++y)
        for (int x = 0; x < A->nx; ++x) {
          size_t i = (size_t)n * np + (size_t)y * A->nx + x;
          psi_g[i] += r[i] / (beta * upwind_diag(A, g, n, x, y));
        }
  }
  free(r);
}

/* One sawtooth cycle for group g with the other groups' scattering frozen in
 * q (Fig. multi_grid_it, Sec. 2.5):
 *   1. r_1 = b - A_PG psi                                    (Eq. Petrov)
 *   2. s_1 = r_1, s_{l+1} = R(s_l)                           (restriction)
 *   3. delta_L = nu upwind Jacobi sweeps from 0 with s_L
 *   4. l = L-1..1: delta_l = nu sweeps from UpSamp(delta_{l+1}) with s_l
 *      (node-block sweeps with scattering on the R14 variant's levels)
 *   5. psi += delta_1
 *   6. one fine PG Jacobi sweep with diagonal beta d_1        (beta = 3)
 * Returns ||r_1||_W / ||q||_W of the input psi (R19).                      */
static double cycle_group(const or_problem* P, int g, double* psi_g, const double* q,
                          double* rn2_out, double* qn2_out) {
  const int L = P->L;
  double* s[OR_MAXLEV];
  double* dl[OR_MAXLEV];
  for (int l = 0; l < L; ++l) {
    s[l] = (double*)calloc(level_size(P, l), sizeof(double));
    dl[l] = (double*)calloc(level_size(P, l), sizeof(double));
  }
  double rn2, qn2;
  group_residual(P, g, psi_g, q, s[0], &rn2, &qn2);
  for (int l = 0; l + 1 < L; ++l) restrict_group(P, l, s[l], s[l + 1]);
  for (int l = L - 1; l >= 0; --l) {
    if (l < L - 1) prolong_group(P, l, dl[l + 1], dl[l]);
    if (scat_on(P, l))
      jacobi_scat_group(P, l, g, s[l], dl[l], P->d.nu);
    else
      jacobi_upwind_group(P, l, g, s[l], dl[l], P->d.nu);
  }
  const size_t n1 = level_size(P, 0);
  for (size_t i = 0; i < n1; ++i) psi_g[i] += dl[0][i];
  pg_jacobi_group(P, g, psi_g, q, 1);
  for (int l = 0; l < L; ++l) {
    free(s[l]);
    free(dl[l]);
  }
  if (rn2_out) *rn2_out = rn2;
  if (qn2_out) *qn2_out = qn2;
  return qn2 > 0 ? sqrt(rn2 / qn2) : sqrt(rn2);
}

/* One multigroup cycle: groups in order (block Gauss-Seidel), one sawtooth
 * cycle each, scattering from the other groups taken from the latest phi.
 * rel_group (nullable, [G]) receives each group's relative residual of its
 * input; the return value is sqrt(sum ||r_g||^2 / sum ||q_g||^2).          */
double or_mg_cycle(const or_problem* P, double* psi, double* rel_group) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny, n1 = level_size(P, 0);
  double* phi = (double*)malloc(sizeof(double) * np * P->G);
  double* q = (double*)malloc(sizeof(double) * np);
  double sr = 0, sq = 0;
  for (int g = 0; g < P->G; ++g) {
    or_scalar_flux(P, psi, phi);
    group_rhs_fixed(P, g, phi, q);
    double rn2, qn2;
    double rel = cycle_group(P, g, psi + (size_t)g * n1, q, &rn2, &qn2);
    if (rel_group) rel_group[g] = rel;
    sr += rn2;
    sq += qn2;
  }
  free(phi);
  free(q);
  return sq > 0 ? sqrt(sr / sq) : sqrt(sr);
}

/* Fine-level smoothing entry points (tests). */
int or_pg_jacobi(const or_problem* P, double* psi, int sweeps) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny, n1 = level_size(P, 0);
  double* phi = (double*)malloc(sizeof(double) * np * P->G);
  double* q = (double*)malloc(sizeof(double) * np);
  for (int g = 0; g < P->G; ++g) {
    or_scalar_flux(P, psi, phi);
    group_rhs_fixed(P, g, phi, q);
    pg_jacobi_group(P, g, psi + (size_t)g * n1, q, sweeps);
  }
  free(phi);
  free(q);
  return 0;
}

/* Relative residual of psi for every group (R19), all groups at once. */
double or_rel_residual(const or_problem* P, const double* psi, double* rel_group) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny, n1 = level_size(P, 0);
  double* phi = (double*)malloc(sizeof(double) * np * P->G);
  double* q = (double*)malloc(sizeof(double) * np);
  double* r = (double*)malloc(sizeof(double) * n1);
  or_scalar_flux(P, psi, phi);
  double sr = 0, sq = 0;
  for (int g = 0; g < P->G; ++g) {
    group_rhs_fixed(P, g, phi, q);
    double rn2, qn2;
    group_residual(P, g, psi + (size_t)g * n1, q, r, &rn2, &qn2);
    if (rel_group) rel_group[g] = qn2 > 0 ? sqrt(rn2 / qn2) : sqrt(rn2);
    sr += rn2;
    sq += qn2;
  }
  free(phi);
  free(q);
  free(r);
  return sq > 0 ? sqrt(sr / sq) : sqrt(sr);
}

/* Fixed-source solve: groups in order; each group is cycled until its
 * relative residual (of the cycle's input) is below rtol.  Groups are
 * revisited (outer passes) until the all-group residual is below rtol or
 * max_outer passes were made (one pass is exact for downscatter only).
 * Returns the number of cycles; *rel_out = final all-group residual.      */
int or_solve(const or_problem* P, double* psi, double rtol, int max_cycles,
             int max_outer, double* rel_out, double* history, int history_len) {
  const or_level* A = &P->lev[0];
  const size_t np = (size_t)A->nx * A->ny, n1 = level_size(P, 0);
  double* phi = (double*)malloc(sizeof(double) * np * P->G);
  double* q = (double*)malloc(sizeof(double) * np);
  int total = 0;
  double rel_all = 0.0;
  if (max_outer < 1) max_outer = 1;
  for (int outer = 0; outer < max_outer; ++outer) {
    for (int g = 0; g < P->G; ++g) {
      or_scalar_flux(P, psi, phi);
      group_rhs_fixed(P, g, phi, q);
      for (int c = 0; c < max_cycles; ++c) {
        double rel = cycle_group(P, g, psi + (size_t)g * n1, q, NULL, NULL);
        if (history && total < history_len) history[total] = rel;
        ++total;
        if (!(rel > rtol)) break; /* also stops on NaN */
      }
    }
    rel_all = or_rel_residual(P, psi, NULL);
    if (rel_all <= rtol || P->G == 1) break;
  }
  if (rel_out) *rel_out = rel_all;
  free(phi);
  free(q);
  return total;
}

int or_omp_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
