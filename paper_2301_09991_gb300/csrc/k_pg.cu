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
#include "btmg_common.cuh"

namespace btmg {
namespace {

constexpr int TX = 32, TY = 32, NT = 256;
constexpr int W6 = TX + 12, H6 = TY + 12;
constexpr int W4 = TX + 8, H4 = TY + 8;
constexpr int W2 = TX + 4, H2 = TY + 4;

template <typename C> struct St {
  // quadratic ConvFEM 1D stencils (offsets -2..2), h = 1
  __device__ __forceinline__ static C m1(int k) {
    return k == 2 ? C(24.0 / 30.0) : ((k == 1 || k == 3) ? C(4.0 / 30.0) : C(-1.0 / 30.0));
  }
  __device__ __forceinline__ static C d1(int k) {
    return k == 0 ? C(1.0 / 12.0) : k == 1 ? C(-8.0 / 12.0) : k == 2 ? C(0) : k == 3 ? C(8.0 / 12.0) : C(-1.0 / 12.0);
  }
  __device__ __forceinline__ static C s1(int k) {
    return k == 2 ? C(30.0 / 12.0) : ((k == 1 || k == 3) ? C(-16.0 / 12.0) : C(1.0 / 12.0));
  }
};

template <typename C> constexpr size_t pg_smem_elems() {
  return (size_t)H6 * W6 + 2 * (size_t)H4 * W6 + 2 * (size_t)H4 * W4 + 2 * (size_t)H2 * W2 +
         5 * (size_t)TY * W2;
}

template <typename C> __device__ __forceinline__ C cmin(C a, C b) { return a < b ? a : b; }
__device__ __forceinline__ float cabs_(float v) { return fabsf(v); }
__device__ __forceinline__ double cabs_(double v) { return fabs(v); }

template <typename T, typename C, int MODE, bool PGON>
__global__ void __launch_bounds__(NT) k_pg(const PgArgs<T, C> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);  // psi_ext, origin (-6,-6), H6 x W6
  C* A = P + H6 * W6;                     // d1_x psi, rows -6.., cols -4.. (H6 x W4)
  C* B = A + H4 * W6;                     // d1_y psi, rows -4.., cols -6.. (H4 x W6)
  C* Px = B + H4 * W6;                    // origin (-4,-4)
  C* Py = Px + H4 * W4;
  C* Kx = Py + H4 * W4;                   // origin (-2,-2)
  C* Ky = Kx + H2 * W2;
  C* U1 = Ky + H2 * W2;                   // rows 0.., cols -2..
  C* U2 = U1 + TY * W2;
  C* V1 = U2 + TY * W2;
  C* V2 = V1 + TY * W2;
  C* V3 = V2 + TY * W2;
  C* Tx = B;   // m1_y Psi_x (rows -2.., cols -4..), B is dead by then
  C* Ty = U1;  // m1_y Psi_y, U1/U2 are not live yet
  C* W1 = A;   // m1_y P (rows 0.., cols -2..), A is dead after stage 2
  __shared__ double red[NT / 32];

  const int tid = threadIdx.x;
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
  const int nx = a.nx, ny = a.ny;
  const size_t npix = (size_t)nx * ny;
  using S = St<C>;

  double nrm = 0.0;
  C phi_acc[(TX * TY) / NT];
#pragma unroll
  for (int k = 0; k < (TX * TY) / NT; ++k) phi_acc[k] = C(0);

  const int n_begin = chunk * a.dpc;
  const int n_end = min(n_begin + a.dpc, a.nd);
  for (int n = n_begin; n < n_end; ++n) {
    const Dir<C> dr = a.dir[n];
    const bool sxp = dr.mu > C(0), syp = dr.nu > C(0);
    const T* psin = a.psi + (size_t)n * npix;
    // ---- stage 0: psi with halo ------------------------------------------
    // Every derivative term (Psi_x, Psi_y, R, k, f^{k-Diff}) is unchanged by
    // a constant shift of psi (all those filters sum to zero), so the PG
    // variant stages psi - c with c = psi at the tile origin: the separable
    // intermediates then round relative to the local variation of psi, not
    // to its magnitude.  sigma_t psi and the update use the unshifted psi.
    const C c0 = PGON ? Conv<T>::ld(psin + (size_t)y0 * nx + x0) : C(0);
    for (int i = tid; i < H6 * W6; i += NT) {
      const int gx = x0 + (i % W6) - 6, gy = y0 + (i / W6) - 6;
      C v;
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny)
        v = Conv<T>::ld(psin + (size_t)gy * nx + gx);
      else if (halo_is_zero(a.bc, gx, gy, nx, ny, sxp, syp))
        v = C(0);
      else
        v = Conv<T>::ld(psin + (size_t)clampi(gy, 0, ny - 1) * nx + clampi(gx, 0, nx - 1));
      P[i] = v - c0;
    }
    __syncthreads();
    if constexpr (PGON) {
    // ---- stage 1: derivative passes first, in difference form ------------
    //   A = d1_x P on rows -6.., cols -4..;  B = d1_y P on rows -4.., cols -6..
    for (int i = tid; i < H6 * W4; i += NT) {
      const int ry = i / W4, rx = i % W4;
      const C* p = P + ry * W6 + rx;
      A[i] = C(8.0 / 12.0) * (p[3] - p[1]) - C(1.0 / 12.0) * (p[4] - p[0]);
    }
    for (int i = tid; i < H4 * W6; i += NT) {
      const int ry = i / W6, cx = i % W6;
      const C* p = P + ry * W6 + cx;
      B[i] = C(8.0 / 12.0) * (p[3 * W6] - p[W6]) - C(1.0 / 12.0) * (p[4 * W6] - p[0]);
    }
    __syncthreads();
    // ---- stage 2: mass passes -> Psi_x = m1_y A / dx, Psi_y = m1_x B / dy -
    for (int i = tid; i < H4 * W4; i += NT) {
      const int ry = i / W4, rx = i % W4;
      C sx = C(0), sy = C(0);
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        sx += S::m1(u) * A[(ry + u) * W4 + rx];
        sy += S::m1(u) * B[ry * W6 + rx + u];
      }
      Px[i] = sx * a.inv_dx;
      Py[i] = sy * a.inv_dy;
    }
    __syncthreads();
    // derived-field halo: nearest interior node
    for (int i = tid; i < H4 * W4; i += NT) {
      const int gx = x0 + (i % W4) - 4, gy = y0 + (i / W4) - 4;
      if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
        const int j = (clampi(gy, 0, ny - 1) - y0 + 4) * W4 + (clampi(gx, 0, nx - 1) - x0 + 4);
        Px[i] = Px[j];
        Py[i] = Py[j];
      }
    }
    __syncthreads();
    // ---- stage 3: R_x, R_y and k_x, k_y on the 2-halo region ------------
    for (int i = tid; i < H2 * W4; i += NT) {
      const int ry = i / W4, cx = i % W4;
      C tx = C(0), ty = C(0);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        tx += S::m1(v) * Px[(ry + v) * W4 + cx];
        ty += S::m1(v) * Py[(ry + v) * W4 + cx];
      }
      Tx[i] = tx;
      Ty[i] = ty;
    }
    __syncthreads();
    {
      const C amu = cabs_(dr.mu), anu = cabs_(dr.nu);
      const C kxmax = a.dx * amu, kymax = a.dy * anu;
      for (int i = tid; i < H2 * W2; i += NT) {
        const int ry = i / W2, rx = i % W2;
        C mx = C(0), my = C(0);
#pragma unroll
        for (int u = 0; u < 5; ++u) {
          mx += S::m1(u) * Tx[ry * W4 + rx + u];
          my += S::m1(u) * Ty[ry * W4 + rx + u];
        }
        const C pxc = Px[(ry + 2) * W4 + rx + 2], pyc = Py[(ry + 2) * W4 + rx + 2];
        const C Rx = a.a_r * dr.mu * (mx - pxc), Ry = a.a_r * dr.nu * (my - pyc);
        const C kxa = a.a_kabs * cabs_(Rx) * a.dx / (a.eps_k + cabs_(pxc));
        const C kya = a.a_kabs * cabs_(Ry) * a.dy / (a.eps_k + cabs_(pyc));
        const C kxs = a.a_ksq * Rx * Rx * a.dx / (a.eps_k + amu * pxc * pxc);
        const C kys = a.a_ksq * Ry * Ry * a.dy / (a.eps_k + anu * pyc * pyc);
        Kx[i] = cmin(cmin(kxmax, kxa), kxs);
        Ky[i] = cmin(cmin(kymax, kya), kys);
      }
    }
    __syncthreads();
    for (int i = tid; i < H2 * W2; i += NT) {
      const int gx = x0 + (i % W2) - 2, gy = y0 + (i / W2) - 2;
      if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
        const int j = (clampi(gy, 0, ny - 1) - y0 + 2) * W2 + (clampi(gx, 0, nx - 1) - x0 + 2);
        Kx[i] = Kx[j];
        Ky[i] = Ky[j];
      }
    }
    __syncthreads();
    // ---- stage 4: y passes of the k-Diff terms ---------------------------
    for (int i = tid; i < TY * W2; i += NT) {
      const int ry = i / W2, rx = i % W2;
      C u1 = C(0), u2 = C(0), w1 = C(0), v1 = C(0), v2 = C(0), v3 = C(0);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const C kx = Kx[(ry + v) * W2 + rx], ky = Ky[(ry + v) * W2 + rx];
        const C p = P[(ry + 4 + v) * W6 + rx + 4];
        u1 += S::m1(v) * kx * p;
        u2 += S::m1(v) * kx;
        w1 += S::m1(v) * p;
        v1 += S::s1(v) * ky * p;
        v2 += S::s1(v) * ky;
        v3 += S::s1(v) * p;
      }
      U1[i] = u1;
      U2[i] = u2;
      W1[i] = w1;
      V1[i] = v1;
      V2[i] = v2;
      V3[i] = v3;
    }
    __syncthreads();
    }  // PGON
    // ---- stage 5: assemble r on the tile ---------------------------------
    T* outn = (MODE == PG_JACOBI) ? a.psi_out + (size_t)n * npix : nullptr;
    C* rn = (MODE == PG_RESID) ? a.r_out + (size_t)n * npix : nullptr;
#pragma unroll
    for (int k = 0; k < (TX * TY) / NT; ++k) {
      const int i = tid + k * NT;
      const int ry = i / TX, rx = i % TX;
      const int gx = x0 + rx, gy = y0 + ry;
      if (gx >= nx || gy >= ny) continue;
      const C pc = P[(ry + 6) * W6 + rx + 6];  // psi - c0
      const size_t gi = (size_t)gy * nx + gx;
      const C psi_c = Conv<T>::ld(psin + gi);  // unshifted psi of this node
      const C sig = a.sigt[gi];
      C Apsi;
      if constexpr (PGON) {
        C fkp = C(0), fp = C(0), fk = C(0), gkp = C(0), gp = C(0), gk = C(0);
#pragma unroll
        for (int u = 0; u < 5; ++u) {
          fkp += S::s1(u) * U1[ry * W2 + rx + u];
          fp += S::s1(u) * W1[ry * W2 + rx + u];
          fk += S::s1(u) * U2[ry * W2 + rx + u];
          gkp += S::m1(u) * V1[ry * W2 + rx + u];
          gp += S::m1(u) * V3[ry * W2 + rx + u];
          gk += S::m1(u) * V2[ry * W2 + rx + u];
        }
        const C kxc = Kx[(ry + 2) * W2 + rx + 2], kyc = Ky[(ry + 2) * W2 + rx + 2];
        const C Dx = (fkp + kxc * fp - pc * fk) * a.inv_dx2;
        const C Dy = (gkp + kyc * gp - pc * gk) * a.inv_dy2;
        Apsi = dr.mu * Px[(ry + 4) * W4 + rx + 4] + dr.nu * Py[(ry + 4) * W4 + rx + 4] +
               a.half * (Dx + Dy) + sig * psi_c;
      } else {
        // upwind filters of Sec. 2.4 (one-sided by the signs of mu and nu)
        const C ux = sxp ? (pc - P[(ry + 6) * W6 + rx + 5]) : (P[(ry + 6) * W6 + rx + 7] - pc);
        const C uy = syp ? (pc - P[(ry + 5) * W6 + rx + 6]) : (P[(ry + 7) * W6 + rx + 6] - pc);
        Apsi = dr.mu * ux * a.inv_dx + dr.nu * uy * a.inv_dy + sig * psi_c;
      }
      const C r = a.b[gi] - Apsi;
      if (MODE == PG_RESID) {
        rn[gi] = r;
        nrm += (double)dr.w * (double)a.dxdy * (double)r * (double)r;
      } else {
        const C d = a.beta * (dr.ax + dr.ay + sig);
        const C pn = psi_c + r / d;
        Conv<T>::st(outn + gi, pn);
        phi_acc[k] += dr.w * stored<T, C>(pn);
      }
    }
    __syncthreads();
  }
  if (MODE == PG_JACOBI) {
    C* ph = a.phi_part + (size_t)chunk * npix;
#pragma unroll
    for (int k = 0; k < (TX * TY) / NT; ++k) {
      const int i = tid + k * NT;
      const int gx = x0 + i % TX, gy = y0 + i / TX;
      if (gx < nx && gy < ny) ph[(size_t)gy * nx + gx] = phi_acc[k];
    }
  } else {
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) red[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      a.norm_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
  }
}

template <typename T, typename C, int MODE, bool PGON>
cudaError_t launch_mode(const PgArgs<T, C>& a, int nchunk, cudaStream_t s) {
  // the upwind variant only needs the psi tile
  const size_t smem = (PGON ? pg_smem_elems<C>() : (size_t)H6 * W6) * sizeof(C);
  static bool attr_set = false;  // per instantiation, once per process
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(k_pg<T, C, MODE, PGON>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tiles_y = (a.ny + TY - 1) / TY;
  dim3 grid(a.tiles_x * tiles_y, nchunk);
  k_pg<T, C, MODE, PGON><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_pg(const PgArgs<T, C>& a, int mode, bool pg, int nchunk, cudaStream_t s) {
  if (pg)
    return mode == PG_RESID ? launch_mode<T, C, PG_RESID, true>(a, nchunk, s)
                            : launch_mode<T, C, PG_JACOBI, true>(a, nchunk, s);
  return mode == PG_RESID ? launch_mode<T, C, PG_RESID, false>(a, nchunk, s)
                          : launch_mode<T, C, PG_JACOBI, false>(a, nchunk, s);
}

template cudaError_t launch_pg<double, double>(const PgArgs<double, double>&, int, bool, int, cudaStream_t);
template cudaError_t launch_pg<float, float>(const PgArgs<float, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_pg<__nv_bfloat16, float>(const PgArgs<__nv_bfloat16, float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_pg<__half, float>(const PgArgs<__half, float>&, int, bool, int, cudaStream_t);

int pg_tile() { return TX; }

}  // namespace btmg
