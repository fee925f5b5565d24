// k_unet.cu -- kernels and host driver of the learned correction: a small
// U-net (4 levels, 16/32/48/64 channels, 3x3 convolutions, average pooling,
// nearest upsampling with skip concatenation) trained and evaluated on the
// GPU by these kernels.  Activations and compute weights are BF16 in NHWC
// layout; accumulation is FP32; master weights and Adam moments are FP32.
//
// Convolutions (forward and input gradient) are implicit GEMMs on the tensor
// cores: M = pixels, N = output channels, K = taps x input channels, with
// mma.sync.m16n8k16 BF16 -> FP32; a warp owns 16 pixels and every output
// channel, the weights of the layer are staged in shared memory.  The weight
// gradient is a deterministic two-stage FP32 reduction over pixels.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/btmg.h"
#include "btmg_common.cuh"

namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------ conv forward --
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Y[p][co] = act(bias[co] + sum_{tap, ci} Wt[co][tap][ci] X[p + off(tap)][ci])
// X: [P][CIN] bf16 (P = N*H*W), CIN % 16 == 0; Wt: [COUT][KS*KS][CIN] bf16;
// COUT % 8 == 0, COUT <= 112.  Zero padding outside the image.
template <int KS>
__global__ void __launch_bounds__(128) k_conv_fwd(const bf16* __restrict__ X, int N, int H, int W, int CIN,
                                                   const bf16* __restrict__ Wt, const float* __restrict__ bias,
                                                   int COUT, bf16* __restrict__ Y, float* __restrict__ Yf,
                                                   int relu) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16* sw = reinterpret_cast<bf16*>(smem_raw);
  const int K = KS * KS * CIN;
  for (int i = threadIdx.x; i < COUT * K / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(sw)[i] = reinterpret_cast<const uint32_t*>(Wt)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long P = (long)N * H * W;
  const long m0 = ((long)blockIdx.x * 4 + warp) * 16;
  if (m0 >= P) return;
  // the two pixels of this lane: rows g and g + 8 of the warp's tile
  long pr[2];
  int py[2], px[2], pn[2];
  bool pv[2];
  for (int h = 0; h < 2; ++h) {
    pr[h] = m0 + g + 8 * h;
    pv[h] = pr[h] < P;
    const long q = pv[h] ? pr[h] : 0;
    px[h] = (int)(q % W);
    py[h] = (int)((q / W) % H);
    pn[h] = (int)(q / ((long)W * H));
  }
  constexpr int MAXNT = 14;
  const int NT = COUT / 8;
  float acc[MAXNT][4];
#pragma unroll
  for (int j = 0; j < MAXNT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int tap = 0; tap < KS * KS; ++tap) {
    const int dy = KS == 3 ? tap / 3 - 1 : 0, dx = KS == 3 ? tap % 3 - 1 : 0;
    const bf16* src[2];
    for (int h = 0; h < 2; ++h) {
      const int yy = py[h] + dy, xx = px[h] + dx;
      const bool ok = pv[h] && yy >= 0 && yy < H && xx >= 0 && xx < W;
      src[h] = ok ? X + (((long)pn[h] * H + yy) * W + xx) * CIN : nullptr;
    }
    for (int kc = 0; kc < CIN; kc += 16) {
      uint32_t a[4];
      a[0] = src[0] ? ld_pair(src[0] + kc + 2 * t) : 0u;
      a[1] = src[1] ? ld_pair(src[1] + kc + 2 * t) : 0u;
      a[2] = src[0] ? ld_pair(src[0] + kc + 8 + 2 * t) : 0u;
      a[3] = src[1] ? ld_pair(src[1] + kc + 8 + 2 * t) : 0u;
      const int kb = tap * CIN + kc;
#pragma unroll
      for (int j = 0; j < MAXNT; ++j) {
        if (j < NT) {
          const bf16* wr = sw + (long)(j * 8 + g) * K + kb;
          mma_bf16(acc[j], a, ld_pair(wr + 2 * t), ld_pair(wr + 8 + 2 * t));
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < MAXNT; ++j) {
    if (j >= NT) continue;
    for (int h = 0; h < 2; ++h) {
      if (!pv[h]) continue;
      const int co = j * 8 + 2 * t;
      float v0 = acc[j][2 * h] + bias[co], v1 = acc[j][2 * h + 1] + bias[co + 1];
      if (relu) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      if (Y) {
        __nv_bfloat162 o;
        o.x = __float2bfloat16_rn(v0);
        o.y = __float2bfloat16_rn(v1);
        *reinterpret_cast<__nv_bfloat162*>(Y + pr[h] * COUT + co) = o;
      }
      if (Yf) {
        Yf[pr[h] * COUT + co] = v0;
        Yf[pr[h] * COUT + co + 1] = v1;
      }
    }
  }
}

// Wf[ci][tap][co] = Wt[co][KS*KS-1-tap][ci]: weights of the input-gradient
// convolution (a convolution with the flipped, transposed kernel).
__global__ void k_flip(const bf16* __restrict__ Wt, int COUT, int KK, int CIN, bf16* __restrict__ Wf) {
  const long n = (long)COUT * KK * CIN;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int co = (int)(i % COUT);
    const int tap = (int)((i / COUT) % KK);
    const int ci = (int)(i / ((long)COUT * KK));
    Wf[i] = Wt[((long)co * KK + (KK - 1 - tap)) * CIN + ci];
  }
}

// ---------------------------------------------------------- weight gradient --
// part[b][co][tap][ci] = sum over the pixels of block b of dY[p][co] X[p+off][ci]
// (block = 64 pixels; 16x16 (co, ci) threads tile the output, all taps).
template <int KS>
__global__ void __launch_bounds__(256) k_conv_dw(const bf16* __restrict__ X, const bf16* __restrict__ dY, int N,
                                                 int H, int W, int CIN, int COUT, float* __restrict__ part,
                                                 float* __restrict__ dbias_part) {
  constexpr int PB = 64;
  __shared__ float sdy[PB][17];
  __shared__ float sx[PB][17];
  const long P = (long)N * H * W;
  const long p0 = (long)blockIdx.x * PB;
  const int tco = threadIdx.x & 15, tci = threadIdx.x >> 4;
  const int KK = KS * KS;
  for (int co0 = 0; co0 < COUT; co0 += 16) {
    // dY tile (pixels x 16 output channels)
    for (int i = threadIdx.x; i < PB * 16; i += 256) {
      const int pp = i / 16, c = i % 16;
      const long p = p0 + pp;
      sdy[pp][c] = (p < P && co0 + c < COUT) ? __bfloat162float(dY[p * COUT + co0 + c]) : 0.f;
    }
    __syncthreads();
    if (dbias_part && tci == 0) {
      float s = 0.f;
      for (int pp = 0; pp < PB; ++pp) s += sdy[pp][tco];
      if (co0 + tco < COUT) dbias_part[(long)blockIdx.x * COUT + co0 + tco] = s;
    }
    for (int tap = 0; tap < KK; ++tap) {
      const int dy = KS == 3 ? tap / 3 - 1 : 0, dx = KS == 3 ? tap % 3 - 1 : 0;
      for (int ci0 = 0; ci0 < CIN; ci0 += 16) {
        __syncthreads();
        for (int i = threadIdx.x; i < PB * 16; i += 256) {
          const int pp = i / 16, c = i % 16;
          const long p = p0 + pp;
          float v = 0.f;
          if (p < P) {
            const int x = (int)(p % W), y = (int)((p / W) % H);
            const long nimg = p / ((long)W * H);
            const int yy = y + dy, xx = x + dx;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
              v = __bfloat162float(X[((nimg * H + yy) * W + xx) * CIN + ci0 + c]);
          }
          sx[pp][c] = v;
        }
        __syncthreads();
        float s = 0.f;
#pragma unroll 8
        for (int pp = 0; pp < PB; ++pp) s += sdy[pp][tco] * sx[pp][tci];
        if (co0 + tco < COUT)
          part[(((long)blockIdx.x * COUT + co0 + tco) * KK + tap) * CIN + ci0 + tci] = s;
      }
    }
    __syncthreads();
  }
}

// out[i] (+)= sum_b part[b][i]  (deterministic)
__global__ void k_reduce_parts(const float* __restrict__ part, int nb, long n, float* __restrict__ out, int add) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(long)b * n + i];
    out[i] = add ? out[i] + s : s;
  }
}

// ------------------------------------------------------------- elementwise --
// dX = dY where Y > 0 (ReLU backward on the stored post-activation output)
__global__ void k_relu_bwd(bf16* __restrict__ dY, const bf16* __restrict__ Y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(Y[i]) > 0.f)) dY[i] = __float2bfloat16_rn(0.f);
}
// 2x2 average pooling, NHWC
__global__ void k_pool_fwd(const bf16* __restrict__ X, int N, int H, int W, int C, bf16* __restrict__ Y) {
  const int H2 = H / 2, W2 = W / 2;
  const long n = (long)N * H2 * W2 * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W2), y = (int)((p / W2) % H2);
    const long b = p / ((long)W2 * H2);
    const bf16* s = X + ((b * H + 2 * y) * W + 2 * x) * C + c;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(long)W * C]) +
                    __bfloat162float(s[(long)W * C + C]);
    Y[i] = __float2bfloat16_rn(0.25f * v);
  }
}
__global__ void k_pool_bwd(const bf16* __restrict__ dY, int N, int H, int W, int C, bf16* __restrict__ dX, int add) {
  const long n = (long)N * H * W * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    const float g = 0.25f * __bfloat162float(dY[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]);
    dX[i] = __float2bfloat16_rn(add ? __bfloat162float(dX[i]) + g : g);
  }
}
// nearest 2x upsampling of X [N][H][W][C] into channels [off, off + C) of
// Y [N][2H][2W][CT] (the skip concatenation writes the other channels)
__global__ void k_up_fwd(const bf16* __restrict__ X, int N, int H, int W, int C, bf16* __restrict__ Y, int CT, int off) {
  const long n = (long)N * 4 * H * W * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % (2 * W)), y = (int)((p / (2 * W)) % (2 * H));
    const long b = p / (4L * W * H);
    Y[p * CT + off + c] = X[((b * H + y / 2) * W + x / 2) * C + c];
  }
}
__global__ void k_up_bwd(const bf16* __restrict__ dY, int N, int H, int W, int C, int CT, int off,
                         bf16* __restrict__ dX) {
  const long n = (long)N * H * W * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    float s = 0.f;
    for (int k = 0; k < 4; ++k) {
      const long q = (b * 2 * H + 2 * y + k / 2) * 2 * W + 2 * x + k % 2;
      s += __bfloat162float(dY[q * CT + off + c]);
    }
    dX[i] = __float2bfloat16_rn(s);
  }
}
// copy channels [0, C) of X [P][C] into channels [off, off + C) of Y [P][CT]
// (fwd), or add channels [off, off + C) of dY into dX [P][C] (bwd)
__global__ void k_chan_copy(const bf16* __restrict__ X, long P, int C, bf16* __restrict__ Y, int CT, int off) {
  const long n = P * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    Y[(i / C) * CT + off + i % C] = X[i];
}
__global__ void k_chan_add(const bf16* __restrict__ dY, long P, int C, int CT, int off, bf16* __restrict__ dX) {
  const long n = P * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dX[i] = __float2bfloat16_rn(__bfloat162float(dX[i]) + __bfloat162float(dY[(i / C) * CT + off + i % C]));
}
// network input: x [P][cin] FP32 -> X [P][16] BF16 (zero padded channels)
__global__ void k_pack_input(const float* __restrict__ x, long P, int cin, bf16* __restrict__ X) {
  const long n = P * 16;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % 16);
    X[i] = __float2bfloat16_rn(c < cin ? x[(i / 16) * cin + c] : 0.f);
  }
}
// output channel 0 of Yf [P][16] -> y [P]
__global__ void k_take0(const float* __restrict__ Yf, long P, float* __restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x)
    y[i] = Yf[i * 16];
}
// MSE loss L = mean (y - t)^2 over P; dY [P][16] (channel 0 = 2 (y - t) / P);
// per-block partial sums of the loss
__global__ void k_mse(const float* __restrict__ Yf, const float* __restrict__ tgt, long P, bf16* __restrict__ dY,
                      double* __restrict__ lpart) {
  __shared__ double red[8];
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
    const float d = Yf[i * 16] - tgt[i];
    acc += (double)d * d;
    for (int c = 0; c < 16; ++c) dY[i * 16 + c] = __float2bfloat16_rn(c == 0 ? 2.f * d / (float)P : 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    lpart[blockIdx.x] = s / (double)P;
  }
}
// Adam on the FP32 master weights, then the BF16 compute copy
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ wb, const unsigned char* __restrict__ frozen,
                       long n, float lr, float b1, float b2, float c1, float c2, float eps) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (frozen[i]) continue;  // padding weights stay zero
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}
__global__ void k_to_bf16(const float* __restrict__ w, bf16* __restrict__ wb, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}
__global__ void k_sum_d(const double* __restrict__ part, int n, double* __restrict__ out) {
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

int gsz(long n) {
  long g = (n + 255) / 256;
  if (g > 152L * 16) g = 152L * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

// ================================================================ host =====
struct ConvL {
  int cin, cout, ks;     // cin, cout as stored (multiples of 16 / 8)
  long woff, boff;       // offsets into the flat parameter vector
  bool relu;
};

struct btmg_unet {
  int in_ch = 3;
  std::vector<ConvL> L;  // order: see build_layers
  long nparam = 0;
  float* w = nullptr;     // FP32 master parameters (weights then biases per layer)
  float* g = nullptr;     // gradients
  float* m = nullptr;
  float* v = nullptr;
  bf16* wb = nullptr;     // BF16 copy (biases unused)
  unsigned char* frozen = nullptr;  // 1 for padding weights (kept 0)
  long step = 0;
  // activation workspace for one (N, H, W)
  int N = 0, H = 0, W = 0;
  std::vector<bf16*> act;  // see forward()
  std::vector<bf16*> grad;
  float* yf = nullptr;     // output conv in FP32 [P][16]
  float* xin = nullptr;
  bf16* wflip = nullptr;   // flipped weights scratch (largest layer)
  float* part = nullptr;   // dW partials
  long part_n = 0;
  float* dbpart = nullptr;
  double* lpart = nullptr;
  double* dloss = nullptr;
  double* hloss = nullptr;
};

namespace {

thread_local std::string u_err;
int uerr(int code, const char* m) {
  u_err = m;
  return code;
}
#define UCK(...)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (__VA_ARGS__);                                                   \
    if (e_ != cudaSuccess) return uerr(BTMG_ERR_CUDA, cudaGetErrorString(e_));        \
  } while (0)

// channel plan: encoder e1 (16) e2 (32) e3 (48), bottleneck (64), decoder
// d3 (48 from 64 + 48), d2 (32 from 48 + 32), d1 (16 from 32 + 16), out 1
void build_layers(btmg_unet* U) {
  const int spec[][4] = {
      // cin, cout, ks, relu
      {16, 16, 3, 1},   // 0 e1a (input padded to 16 channels)
      {16, 16, 3, 1},   // 1 e1b
      {16, 32, 3, 1},   // 2 e2a
      {32, 32, 3, 1},   // 3 e2b
      {32, 48, 3, 1},   // 4 e3a
      {48, 48, 3, 1},   // 5 e3b
      {48, 64, 3, 1},   // 6 ba
      {64, 64, 3, 1},   // 7 bb
      {112, 48, 3, 1},  // 8 d3 (cat e3 48 + up(b) 64)
      {80, 32, 3, 1},   // 9 d2 (cat e2 32 + up(d3) 48)
      {48, 16, 3, 1},   // 10 d1 (cat e1 16 + up(d2) 32)
      {16, 16, 1, 0},   // 11 out (1 real output channel)
  };
  long off = 0;
  for (auto& s : spec) {
    ConvL c;
    c.cin = s[0];
    c.cout = s[1];
    c.ks = s[2];
    c.relu = s[3] != 0;
    c.woff = off;
    off += (long)c.cout * c.ks * c.ks * c.cin;
    c.boff = off;
    off += c.cout;
    U->L.push_back(c);
  }
  U->nparam = off;
}

bool is_padding(const btmg_unet* U, long i) {
  // input channels >= in_ch of layer 0, output channels >= 1 of layer 11
  const ConvL& c0 = U->L[0];
  if (i >= c0.woff && i < c0.boff) {
    const long r = (i - c0.woff) % c0.cin;
    return r >= U->in_ch;
  }
  const ConvL& c11 = U->L[11];
  if (i >= c11.woff && i < c11.boff) return (i - c11.woff) / ((long)c11.ks * c11.ks * c11.cin) >= 1;
  if (i >= c11.boff && i < c11.boff + c11.cout) return i - c11.boff >= 1;
  return false;
}

void free_ws(btmg_unet* U) {
  for (auto p : U->act) cudaFree(p);
  for (auto p : U->grad) cudaFree(p);
  U->act.clear();
  U->grad.clear();
  for (void* p : {(void*)U->yf, (void*)U->xin, (void*)U->wflip, (void*)U->part, (void*)U->dbpart,
                  (void*)U->lpart, (void*)U->dloss})
    if (p) cudaFree(p);
  U->yf = U->xin = nullptr;
  U->wflip = nullptr;
  U->part = U->dbpart = nullptr;
  U->lpart = U->dloss = nullptr;
  U->N = U->H = U->W = 0;
}

// activation buffers (index: channels at resolution):
//  0 x16 (P0,16)  1 e1a (P0,16) 2 e1 (P0,16)  3 p1 (P1,16)  4 e2a (P1,32) 5 e2 (P1,32)
//  6 p2 (P2,32)   7 e3a (P2,48) 8 e3 (P2,48)  9 p3 (P3,48) 10 ba (P3,64) 11 b (P3,64)
// 12 c3 (P2,112) 13 d3 (P2,48) 14 c2 (P1,80)  15 d2 (P1,32) 16 c1 (P0,48) 17 d1 (P0,16)
// 18 dout (P0,16) (gradient of the output only)
int ensure_ws(btmg_unet* U, int N, int H, int W) {
  // kernel attributes once per process, outside any graph capture (the
  // first forward call of a size runs eagerly)
  static bool attrs = false;
  if (!attrs) {
    UCK(cudaFuncSetAttribute(k_conv_fwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    UCK(cudaFuncSetAttribute(k_conv_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attrs = true;
  }
  if (U->N == N && U->H == H && U->W == W) return BTMG_OK;
  free_ws(U);
  const long P0 = (long)N * H * W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  const long sz[19][2] = {{P0, 16}, {P0, 16}, {P0, 16}, {P1, 16}, {P1, 32}, {P1, 32}, {P2, 32},
                          {P2, 48}, {P2, 48}, {P3, 48}, {P3, 64}, {P3, 64}, {P2, 112}, {P2, 48},
                          {P1, 80}, {P1, 32}, {P0, 48}, {P0, 16}, {P0, 16}};
  for (auto& s : sz) {
    bf16 *a = nullptr, *g = nullptr;
    UCK(cudaMalloc(&a, sizeof(bf16) * s[0] * s[1]));
    UCK(cudaMalloc(&g, sizeof(bf16) * s[0] * s[1]));
    U->act.push_back(a);
    U->grad.push_back(g);
  }
  UCK(cudaMalloc(&U->yf, sizeof(float) * P0 * 16));
  UCK(cudaMalloc(&U->xin, sizeof(float) * P0 * 16));
  long maxw = 0;
  for (auto& c : U->L) maxw = std::max(maxw, (long)c.cout * c.ks * c.ks * c.cin);
  UCK(cudaMalloc(&U->wflip, sizeof(bf16) * maxw));
  const long nb0 = (P0 + 63) / 64;
  U->part_n = nb0 * maxw;
  UCK(cudaMalloc(&U->part, sizeof(float) * U->part_n));
  UCK(cudaMalloc(&U->dbpart, sizeof(float) * nb0 * 112));
  UCK(cudaMalloc(&U->lpart, sizeof(double) * 2048));
  UCK(cudaMalloc(&U->dloss, sizeof(double)));
  U->N = N;
  U->H = H;
  U->W = W;
  return BTMG_OK;
}

cudaError_t conv(btmg_unet* U, int li, const bf16* X, long N, int H, int W, bf16* Y, float* Yf, const bf16* wt,
                 int cin, int cout, cudaStream_t s) {
  const ConvL& c = U->L[li];
  const long P = N * H * W;
  const int KK = c.ks * c.ks;
  const size_t smem = sizeof(bf16) * (size_t)cout * KK * cin;
  const int blocks = (int)((P + 63) / 64);
  const int relu = (Y == nullptr) ? 0 : (c.relu ? 1 : 0);
  if (c.ks == 3) {
    k_conv_fwd<3><<<blocks, 128, smem, s>>>(X, (int)N, H, W, cin, wt, U->w + c.boff, cout, Y, Yf, relu);
  } else {
    k_conv_fwd<1><<<blocks, 128, smem, s>>>(X, (int)N, H, W, cin, wt, U->w + c.boff, cout, Y, Yf, relu);
  }
  return cudaGetLastError();
}

// forward pass; keeps every activation for the backward pass
int forward(btmg_unet* U, const float* x, int N, int H, int W, cudaStream_t s) {
  if (int rc = ensure_ws(U, N, H, W)) return rc;
  auto& A = U->act;
  const long P0 = (long)N * H * W;
  k_pack_input<<<gsz(P0 * 16), 256, 0, s>>>(x, P0, U->in_ch, A[0]);
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  auto cv = [&](int li, const bf16* X, int h, int w, bf16* Y) {
    const ConvL& c = U->L[li];
    return conv(U, li, X, N, h, w, Y, nullptr, U->wb + c.woff, c.cin, c.cout, s);
  };
  UCK(cv(0, A[0], H, W, A[1]));
  UCK(cv(1, A[1], H, W, A[2]));
  k_pool_fwd<<<gsz(P0 / 4 * 16), 256, 0, s>>>(A[2], N, H, W, 16, A[3]);
  UCK(cv(2, A[3], H1, W1, A[4]));
  UCK(cv(3, A[4], H1, W1, A[5]));
  k_pool_fwd<<<gsz(P0 / 16 * 32), 256, 0, s>>>(A[5], N, H1, W1, 32, A[6]);
  UCK(cv(4, A[6], H2, W2, A[7]));
  UCK(cv(5, A[7], H2, W2, A[8]));
  k_pool_fwd<<<gsz(P0 / 64 * 48), 256, 0, s>>>(A[8], N, H2, W2, 48, A[9]);
  UCK(cv(6, A[9], H3, W3, A[10]));
  UCK(cv(7, A[10], H3, W3, A[11]));
  // decoder: cat(skip, up(coarse))
  k_chan_copy<<<gsz(P0 / 16 * 48), 256, 0, s>>>(A[8], P0 / 16, 48, A[12], 112, 0);
  k_up_fwd<<<gsz(P0 / 16 * 64), 256, 0, s>>>(A[11], N, H3, W3, 64, A[12], 112, 48);
  UCK(cv(8, A[12], H2, W2, A[13]));
  k_chan_copy<<<gsz(P0 / 4 * 32), 256, 0, s>>>(A[5], P0 / 4, 32, A[14], 80, 0);
  k_up_fwd<<<gsz(P0 / 4 * 48), 256, 0, s>>>(A[13], N, H2, W2, 48, A[14], 80, 32);
  UCK(cv(9, A[14], H1, W1, A[15]));
  k_chan_copy<<<gsz(P0 * 16), 256, 0, s>>>(A[2], P0, 16, A[16], 48, 0);
  k_up_fwd<<<gsz(P0 * 32), 256, 0, s>>>(A[15], N, H1, W1, 32, A[16], 48, 16);
  UCK(cv(10, A[16], H, W, A[17]));
  {
    const ConvL& c = U->L[11];
    UCK(conv(U, 11, A[17], N, H, W, nullptr, U->yf, U->wb + c.woff, c.cin, c.cout, s));
  }
  UCK(cudaGetLastError());
  return BTMG_OK;
}

// backward of conv li: input X (forward input), output Y (post-activation,
// or nullptr for the linear output layer), dY (gradient of Y; modified in
// place by the ReLU mask); writes dW/db into U->g and dX (nullable)
int conv_bwd(btmg_unet* U, int li, const bf16* X, const bf16* Y, bf16* dY, long N, int H, int W, bf16* dX,
             cudaStream_t s) {
  const ConvL& c = U->L[li];
  const long P = N * H * W;
  const int KK = c.ks * c.ks;
  if (Y && c.relu) k_relu_bwd<<<gsz(P * c.cout), 256, 0, s>>>(dY, Y, P * c.cout);
  const int nb = (int)((P + 63) / 64);
  const long nw = (long)c.cout * KK * c.cin;
  if (c.ks == 3)
    k_conv_dw<3><<<nb, 256, 0, s>>>(X, dY, (int)N, H, W, c.cin, c.cout, U->part, U->dbpart);
  else
    k_conv_dw<1><<<nb, 256, 0, s>>>(X, dY, (int)N, H, W, c.cin, c.cout, U->part, U->dbpart);
  k_reduce_parts<<<gsz(nw), 256, 0, s>>>(U->part, nb, nw, U->g + c.woff, 0);
  k_reduce_parts<<<gsz(c.cout), 256, 0, s>>>(U->dbpart, nb, c.cout, U->g + c.boff, 0);
  if (dX) {
    // dX = conv(dY, flipped transposed weights), no bias, no activation
    k_flip<<<gsz(nw), 256, 0, s>>>(U->wb + c.woff, c.cout, KK, c.cin, U->wflip);
    const size_t smem = sizeof(bf16) * (size_t)c.cin * KK * c.cout;
    const int blocks = (int)((P + 63) / 64);
    // the forward kernel adds bias[co]: give it the zero tail of yf as bias
    UCK(cudaMemsetAsync(U->xin, 0, sizeof(float) * 128, s));
    if (c.ks == 3) {
        k_conv_fwd<3><<<blocks, 128, smem, s>>>(dY, (int)N, H, W, c.cout, U->wflip, U->xin, c.cin, dX, nullptr, 0);
    } else {
        k_conv_fwd<1><<<blocks, 128, smem, s>>>(dY, (int)N, H, W, c.cout, U->wflip, U->xin, c.cin, dX, nullptr, 0);
    }
  }
  UCK(cudaGetLastError());
  return BTMG_OK;
}

int backward(btmg_unet* U, const float* tgt, cudaStream_t s, double* loss_host) {
  auto& A = U->act;
  auto& D = U->grad;
  const long N = U->N;
  const int H = U->H, W = U->W;
  const long P0 = N * H * W;
  const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
  const int lb = std::min(gsz(P0), 2048);
  k_mse<<<lb, 256, 0, s>>>(U->yf, tgt, P0, D[18], U->lpart);
  k_sum_d<<<1, 1024, 0, s>>>(U->lpart, lb, U->dloss);
  // output layer (linear): d1 grad
  if (int rc = conv_bwd(U, 11, A[17], nullptr, D[18], N, H, W, D[17], s)) return rc;
  if (int rc = conv_bwd(U, 10, A[16], A[17], D[17], N, H, W, D[16], s)) return rc;
  // split c1 = cat(e1, up(d2)): d e1 <- slice, d d2 <- up_bwd(slice)
  k_up_bwd<<<gsz(P0 / 4 * 32), 256, 0, s>>>(D[16], N, H1, W1, 32, 48, 16, D[15]);
  if (int rc = conv_bwd(U, 9, A[14], A[15], D[15], N, H1, W1, D[14], s)) return rc;
  k_up_bwd<<<gsz(P0 / 16 * 48), 256, 0, s>>>(D[14], N, H2, W2, 48, 80, 32, D[13]);
  if (int rc = conv_bwd(U, 8, A[12], A[13], D[13], N, H2, W2, D[12], s)) return rc;
  k_up_bwd<<<gsz(P0 / 64 * 64), 256, 0, s>>>(D[12], N, H3, W3, 64, 112, 48, D[11]);
  if (int rc = conv_bwd(U, 7, A[10], A[11], D[11], N, H3, W3, D[10], s)) return rc;
  if (int rc = conv_bwd(U, 6, A[9], A[10], D[10], N, H3, W3, D[9], s)) return rc;
  // e3 feeds the pool and the concatenation
  k_pool_bwd<<<gsz(P0 / 16 * 48), 256, 0, s>>>(D[9], N, H2, W2, 48, D[8], 0);
  k_chan_add<<<gsz(P0 / 16 * 48), 256, 0, s>>>(D[12], P0 / 16, 48, 112, 0, D[8]);
  if (int rc = conv_bwd(U, 5, A[7], A[8], D[8], N, H2, W2, D[7], s)) return rc;
  if (int rc = conv_bwd(U, 4, A[6], A[7], D[7], N, H2, W2, D[6], s)) return rc;
  k_pool_bwd<<<gsz(P0 / 4 * 32), 256, 0, s>>>(D[6], N, H1, W1, 32, D[5], 0);
  k_chan_add<<<gsz(P0 / 4 * 32), 256, 0, s>>>(D[14], P0 / 4, 32, 80, 0, D[5]);
  if (int rc = conv_bwd(U, 3, A[4], A[5], D[5], N, H1, W1, D[4], s)) return rc;
  if (int rc = conv_bwd(U, 2, A[3], A[4], D[4], N, H1, W1, D[3], s)) return rc;
  k_pool_bwd<<<gsz(P0 * 16), 256, 0, s>>>(D[3], N, H, W, 16, D[2], 0);
  k_chan_add<<<gsz(P0 * 16), 256, 0, s>>>(D[16], P0, 16, 48, 0, D[2]);
  if (int rc = conv_bwd(U, 1, A[1], A[2], D[2], N, H, W, D[1], s)) return rc;
  if (int rc = conv_bwd(U, 0, A[0], A[1], D[1], N, H, W, nullptr, s)) return rc;
  if (loss_host) {
    UCK(cudaMemcpyAsync(U->hloss, U->dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
    UCK(cudaStreamSynchronize(s));
    *loss_host = *U->hloss;
  }
  UCK(cudaGetLastError());
  return BTMG_OK;
}

}  // namespace

extern "C" {

int btmg_unet_create(int32_t in_channels, uint64_t seed, btmg_unet** out) {
  if (!out || in_channels < 1 || in_channels > 16) return uerr(BTMG_ERR_INVALID_ARG, "bad unet arguments");
  *out = nullptr;
  btmg_unet* U = new btmg_unet();
  U->in_ch = in_channels;
  build_layers(U);
  const long n = U->nparam;
  std::vector<float> h(n, 0.f);
  std::vector<unsigned char> fr(n, 0);
  // He-normal initialisation from a splitmix64 stream (host), biases 0
  uint64_t st = seed ? seed : 0x9e3779b97f4a7c15ull;
  auto next = [&]() {
    st += 0x9e3779b97f4a7c15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  };
  auto unif = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  for (size_t li = 0; li < U->L.size(); ++li) {
    const ConvL& c = U->L[li];
    const int fan_in = c.ks * c.ks * (li == 0 ? in_channels : c.cin);
    const double sd = std::sqrt(2.0 / fan_in) * (li == 11 ? 0.1 : 1.0);
    for (long i = c.woff; i < c.boff; ++i) {
      const double u1 = unif(), u2 = unif();
      h[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  for (long i = 0; i < n; ++i)
    if (is_padding(U, i)) {
      h[i] = 0.f;
      fr[i] = 1;
    }
  if (cudaMalloc(&U->w, sizeof(float) * n) != cudaSuccess || cudaMalloc(&U->g, sizeof(float) * n) != cudaSuccess ||
      cudaMalloc(&U->m, sizeof(float) * n) != cudaSuccess || cudaMalloc(&U->v, sizeof(float) * n) != cudaSuccess ||
      cudaMalloc(&U->wb, sizeof(bf16) * n) != cudaSuccess || cudaMalloc(&U->frozen, n) != cudaSuccess ||
      cudaMallocHost(&U->hloss, sizeof(double)) != cudaSuccess) {
    delete U;
    return uerr(BTMG_ERR_OOM, "unet allocation");
  }
  cudaMemcpy(U->w, h.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(U->frozen, fr.data(), n, cudaMemcpyHostToDevice);
  cudaMemset(U->g, 0, sizeof(float) * n);
  cudaMemset(U->m, 0, sizeof(float) * n);
  cudaMemset(U->v, 0, sizeof(float) * n);
  k_to_bf16<<<gsz(n), 256>>>(U->w, U->wb, n);
  if (cudaDeviceSynchronize() != cudaSuccess) return uerr(BTMG_ERR_CUDA, "unet init");
  *out = U;
  return BTMG_OK;
}

int btmg_unet_destroy(btmg_unet* U) {
  if (!U) return BTMG_OK;
  free_ws(U);
  for (void* p : {(void*)U->w, (void*)U->g, (void*)U->m, (void*)U->v, (void*)U->wb, (void*)U->frozen})
    if (p) cudaFree(p);
  if (U->hloss) cudaFreeHost(U->hloss);
  delete U;
  return BTMG_OK;
}

int btmg_unet_num_params(const btmg_unet* U, int64_t* n) {
  if (!U || !n) return uerr(BTMG_ERR_INVALID_ARG, "null argument");
  *n = U->nparam;
  return BTMG_OK;
}

int btmg_unet_get_params(const btmg_unet* U, float* host, int64_t n) {
  if (!U || !host || n != U->nparam) return uerr(BTMG_ERR_INVALID_ARG, "bad parameter buffer");
  UCK(cudaMemcpy(host, U->w, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return BTMG_OK;
}

int btmg_unet_set_params(btmg_unet* U, const float* host, int64_t n) {
  if (!U || !host || n != U->nparam) return uerr(BTMG_ERR_INVALID_ARG, "bad parameter buffer");
  UCK(cudaMemcpy(U->w, host, sizeof(float) * n, cudaMemcpyHostToDevice));
  k_to_bf16<<<gsz(n), 256>>>(U->w, U->wb, n);
  UCK(cudaDeviceSynchronize());
  return BTMG_OK;
}

int btmg_unet_get_grads(const btmg_unet* U, float* host, int64_t n) {
  if (!U || !host || n != U->nparam) return uerr(BTMG_ERR_INVALID_ARG, "bad gradient buffer");
  UCK(cudaMemcpy(host, U->g, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return BTMG_OK;
}

int btmg_unet_forward(btmg_unet* U, const float* x, float* y, int32_t N, int32_t H, int32_t W, void* stream) {
  if (!U || !x || !y || N < 1 || H < 8 || W < 8 || H % 8 || W % 8)
    return uerr(BTMG_ERR_INVALID_ARG, "unet input must be N x H x W with H, W multiples of 8");
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = forward(U, x, N, H, W, s)) return rc;
  const long P = (long)N * H * W;
  k_take0<<<gsz(P), 256, 0, s>>>(U->yf, P, y);
  UCK(cudaGetLastError());
  return BTMG_OK;
}

int btmg_unet_train_step(btmg_unet* U, const float* x, const float* target, int32_t N, int32_t H, int32_t W,
                         float lr, double* loss, void* stream) {
  if (!U || !x || !target || N < 1 || H < 8 || W < 8 || H % 8 || W % 8)
    return uerr(BTMG_ERR_INVALID_ARG, "unet input must be N x H x W with H, W multiples of 8");
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = forward(U, x, N, H, W, s)) return rc;
  if (int rc = backward(U, target, s, loss)) return rc;
  if (lr > 0.f) {
    U->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)U->step), c2 = 1.f - std::pow(b2, (float)U->step);
    k_adam<<<gsz(U->nparam), 256, 0, s>>>(U->w, U->g, U->m, U->v, U->wb, U->frozen, U->nparam, lr, b1, b2, c1, c2,
                                         1e-8f);
  }
  UCK(cudaGetLastError());
  return BTMG_OK;
}

const char* btmg_unet_last_error(void) { return u_err.c_str(); }

}  // extern "C"

// input channels of a U-net (library-internal, used by btmg_set_learned)
int unet_in_channels(const btmg_unet* U) { return U ? U->in_ch : 0; }
