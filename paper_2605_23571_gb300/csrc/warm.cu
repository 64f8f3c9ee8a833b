// Learned warm start (not in the paper): a periodic 1-D convolutional network
// mapping (member right-hand side b_j, control solution dz_0) to a guess of
// the member solution dz_j, used only as the initial iterate of the PCG,
// which then runs to the same tolerance.
//
// Network: 2 -> H -> H -> H -> 1 channels, kernel 5 (tap t reads position
// i + t - 2 mod n), GELU after the first three layers; inputs scaled by the
// training-set RMS of b and dz_0; guess = dz_0 + s_z * out.  Weights are FP32
// masters used as BF16 in every product, activations and accumulation FP32.
// Hand-written kernels: forward convolution (register-blocked 4 channels x 4
// positions per thread, or, for the 64 -> 64 layers, an implicit GEMM on the
// tcgen05 tensor cores), the data gradient as a forward convolution with the
// transposed and flipped kernel, the weight gradient by per-CTA partial sums,
// GELU, MSE and AdamW.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "tc.h"

namespace {

constexpr int KS = 5;       // kernel size
constexpr int TP = 64;      // positions per CTA tile
constexpr int MAXC = 64;    // channel capacity of the kernels

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// out[s][o][i] = bias[o] + sum_{c,t} W[o][c][t] x[s][c][(i + t - 2) mod n];
// pre (if set) keeps the sum, out gets GELU of it when act != 0.
// Grid (S, ceil(n / TP)); 256 threads, each 4 output channels x 4 positions.
__global__ void __launch_bounds__(256) conv_fwd_kernel(int n, int cin, int cout, const float* __restrict__ x,
                                                       const __nv_bfloat16* __restrict__ W,
                                                       const float* __restrict__ bias, float* pre, float* out,
                                                       int act) {
  // dynamic shared memory: input tile [cin][TP + 4] (FP32), weights (BF16)
  extern __shared__ __align__(16) unsigned char wsm_raw[];
  float(*xs)[TP + KS - 1] = reinterpret_cast<float(*)[TP + KS - 1]>(wsm_raw);
  __nv_bfloat16* ws = reinterpret_cast<__nv_bfloat16*>(wsm_raw + (size_t)cin * (TP + KS - 1) * sizeof(float));
  const int s = blockIdx.x, i0 = blockIdx.y * TP;
  const float* xsmp = x + (long long)s * cin * n;
  for (int e = threadIdx.x; e < cin * (TP + KS - 1); e += blockDim.x) {
    const int c = e / (TP + KS - 1), j = e % (TP + KS - 1);
    int g = i0 + j - KS / 2;
    g = (g % n + n) % n;
    xs[c][j] = xsmp[(long long)c * n + g];
  }
  for (int e = threadIdx.x; e < cout * cin * KS; e += blockDim.x) ws[e] = W[e];
  __syncthreads();
  const int ob = (threadIdx.x >> 4) * 4;  // 16 groups of 4 output channels
  const int pb = (threadIdx.x & 15) * 4;  // 16 groups of 4 positions
  if (ob >= cout) return;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int c = 0; c < cin; ++c) {
    float xv[4 + KS - 1];
#pragma unroll
    for (int j = 0; j < 4 + KS - 1; ++j) xv[j] = xs[c][pb + j];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (ob + a < cout) {
        const __nv_bfloat16* wr = ws + ((ob + a) * cin + c) * KS;
#pragma unroll
        for (int t = 0; t < KS; ++t) {
          const float wv = __bfloat162float(wr[t]);
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wv, xv[b + t], acc[a][b]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int o = ob + a;
    if (o >= cout) continue;
    const float bo = bias ? bias[o] : 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + pb + b;
      if (i >= n) continue;
      const float z = acc[a][b] + bo;
      const long long idx = ((long long)s * cout + o) * n + i;
      if (pre) pre[idx] = z;
      out[idx] = act ? gelu_f(z) : z;
    }
  }
}

// ------------------------------------------------ tensor-core convolution
// The 64 -> 64 layers as an implicit GEMM on the tensor cores: for a tile of
// 128 positions, D (128 positions x 64 output channels) = sum over the five
// taps t of A_t (positions x 64 input channels) B_t (64 x 64).  The input
// tile is staged once, 132 rows (positions i0 - 2 .. i0 + 129, periodic),
// each row's 64 channels as eight 16-byte groups, and kept row-contiguous
// within each group of 8 channels: A_t is then A_0 shifted by t rows, a
// descriptor start 16 t bytes further.  Activations stay FP32 in value: each
// is split exactly into three BF16 parts (hi = bf16(x), mid = bf16(x - hi),
// lo = bf16(x - hi - mid); 3 x 8 significant bits), so that the three MMAs
// per step multiply FP32 activations by the BF16 weights exactly, with FP32
// accumulation.  The weights arrive pre-tiled (weights_tile_kernel) by one
// bulk asynchronous copy.
constexpr int kTcPos = 128;               // positions per tile (the MMA's M)
constexpr int kTcRows = kTcPos + KS - 1;  // staged rows
constexpr int kTcRowsP = 136;             // staged rows rounded up to whole core matrices
constexpr int kTcCh = 64;                 // channels in and out
constexpr uint32_t kTcGroup = kTcRowsP * 16;             // bytes of one 8-channel group of a part
constexpr uint32_t kTcPart = (kTcCh / 8) * kTcGroup;      // bytes of one BF16 part of the tile
constexpr uint32_t kTcTap = kTcCh * kTcCh * 2;           // bytes of one tap's weight tile
constexpr size_t kTcSmem = 3 * (size_t)kTcPart + KS * (size_t)kTcTap + 32;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b, __nv_bfloat16* ra, __nv_bfloat16* rb) {
  *ra = __float2bfloat16_rn(a);
  *rb = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(*ra) | ((uint32_t)__bfloat16_as_ushort(*rb) << 16);
}

// out[s][o][i] = bias[o] + sum_{c,t} W[o][c][t] x[s][c][(i + t - 2) mod n]
// (pre and GELU as conv_fwd_kernel) for cin = cout = 64.  Grid (S,
// ceil(n / 128)); 128 threads (warp w reads TMEM lanes 32w.., the tile's
// positions).  Shared: three parts of the staged tile | the five tap tiles
// | two mbarriers (weights copy, MMAs) | TMEM slot.  A bounded wait that
// gives up sets *timeout and the CTA skips its outputs.
__global__ void __launch_bounds__(128) conv_tc_kernel(int n, const float* __restrict__ x,
                                                      const __nv_bfloat16* __restrict__ Wtile,
                                                      const float* __restrict__ bias, float* pre, float* out, int act,
                                                      int* timeout) {
  using namespace eda::tc;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* Apart = tsm;  // part q at q * kTcPart
  unsigned char* Bt = tsm + 3 * kTcPart;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bt + KS * kTcTap);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
  const uint32_t bw = smem_u32(bars), bm = smem_u32(bars + 1);
  const int s = blockIdx.x, i0 = blockIdx.y * kTcPos;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bw) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bm) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bw), "r"((uint32_t)(KS * kTcTap))
                 : "memory");
    bulk_g2s(smem_u32(Bt), Wtile, KS * kTcTap, bw);
  }
  // the tile: item (group g of 8 channels, row j) -> one 16-byte row of each part
  const float* xs = x + (long long)s * kTcCh * n;
  for (int idx = threadIdx.x; idx < (kTcCh / 8) * kTcRows; idx += blockDim.x) {
    const int g = idx / kTcRows, j = idx - g * kTcRows;
    int p = i0 + j - KS / 2;
    p = (p % n + n) % n;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = xs[(long long)(8 * g + e) * n + p];
    uint32_t w3[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      __nv_bfloat16 h0, h1, m0, m1, l0, l1;
      w3[0][e / 2] = pack_bf16(v[e], v[e + 1], &h0, &h1);
      const float r0 = v[e] - __bfloat162float(h0), r1 = v[e + 1] - __bfloat162float(h1);
      w3[1][e / 2] = pack_bf16(r0, r1, &m0, &m1);
      w3[2][e / 2] = pack_bf16(r0 - __bfloat162float(m0), r1 - __bfloat162float(m1), &l0, &l1);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      *reinterpret_cast<uint4*>(Apart + q * kTcPart + g * kTcGroup + j * 16) =
          make_uint4(w3[q][0], w3[q][1], w3[q][2], w3[q][3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint32_t tbase = tmem_alloc(slot, kTcCh);  // includes the block barrier
  if (threadIdx.x == 0) {
    bool have = mbar_wait(bw, 0);
    if (have) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t id = idesc_bf16(kTcCh);
      bool first = true;
      for (int t = 0; t < KS; ++t)
        for (int ks = 0; ks < kTcCh / 16; ++ks) {
          // B_t: 64 output channels x 64 input channels, K-major core matrices
          // (lbo 128 along K, sbo 1024 along N)
          const uint64_t bd = kmajor_desc(smem_u32(Bt + t * kTcTap) + ks * 256u, 128u, 1024u);
          for (int q = 0; q < 3; ++q) {
            // A_t: rows shifted by t; groups of 8 channels kTcGroup apart
            const uint64_t ad = kmajor_desc(smem_u32(Apart + q * kTcPart) + 2u * ks * kTcGroup + 16u * t, kTcGroup,
                                            128u);
            mma_bf16(tbase, ad, bd, id, first ? 0u : 1u);
            first = false;
          }
        }
      mma_commit(bm);
    } else {
      mbar_arrive(bm);
      if (timeout != nullptr) atomicExch(timeout, 1);
    }
    slot[1] = have ? 1u : 0u;
  }
  __syncwarp();
  bool ok = mbar_wait(bm, 0);
  ok = __syncthreads_and(ok ? 1 : 0) != 0 && slot[1] != 0u;
  if (!ok) {
    if (threadIdx.x == 0 && timeout != nullptr) atomicExch(timeout, 1);
    mbar_wait(bw, 0);
    mbar_wait(bm, 0);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = i0 + 32 * w + lane;  // TMEM lane = row = position
    for (int c0 = 0; c0 < kTcCh; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
      if (i < n) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int o = c0 + e;
          const float z = v[e] + (bias ? bias[o] : 0.f);
          const long long idx = ((long long)s * kTcCh + o) * n + i;
          if (pre) pre[idx] = z;
          out[idx] = act ? gelu_f(z) : z;
        }
      }
    }
  }
  tmem_free(tbase, kTcCh);
}

// Tap tiles of a 64 x 64 layer for conv_tc_kernel: forward Tf[t] = W[.][.][t]
// (rows output channel o, K input channel c) and the data gradient's
// Tb[t'] = W[.][.][4 - t'] transposed (rows c, K o), BF16, each tap a 64 x 64
// block of K-major core matrices (core (r / 8, k / 8) at ((r / 8) * 8 +
// k / 8) * 128 bytes, row r % 8 at 16 (r % 8)).
__global__ void weights_tile_kernel(const float* W, __nv_bfloat16* Tf, __nv_bfloat16* Tb) {
  const int total = KS * kTcCh * kTcCh;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int o = e / (kTcCh * KS), c = (e / KS) % kTcCh, t = e % KS;
    const __nv_bfloat16 b = __float2bfloat16_rn(W[e]);
    auto at = [](int r, int k) { return ((((r >> 3) * 8 + (k >> 3)) << 7) + ((r & 7) << 4)) / 2 + (k & 7); };
    Tf[t * kTcCh * kTcCh + at(o, c)] = b;
    Tb[(KS - 1 - t) * kTcCh * kTcCh + at(c, o)] = b;
  }
}

// dW[o][c][t] += sum_{s in slice, i} g[s][o][i] x[s][c][(i + t - 2) mod n],
// db[o] += sum g.  Grid (ceil(cout/16), slices); 256 threads: thread ->
// input channel c = tid / 4 and 4 output channels, 5 taps each.
__global__ void __launch_bounds__(256) conv_wgrad_kernel(int n, int S, int cin, int cout, const float* __restrict__ x,
                                                         const float* __restrict__ g, float* dW, float* db) {
  constexpr int CH = 128;
  __shared__ float xs[MAXC][CH + KS - 1];
  __shared__ float gs[16][CH];
  const int o0 = blockIdx.x * 16;
  const int c = threadIdx.x >> 2, os = (threadIdx.x & 3) * 4;
  float acc[4][KS];
  float bacc[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    bacc[a] = 0.f;
#pragma unroll
    for (int t = 0; t < KS; ++t) acc[a][t] = 0.f;
  }
  for (int s = blockIdx.y; s < S; s += gridDim.y) {
    const float* xsmp = x + (long long)s * cin * n;
    const float* gsmp = g + (long long)s * cout * n;
    for (int i0 = 0; i0 < n; i0 += CH) {
      __syncthreads();
      for (int e = threadIdx.x; e < cin * (CH + KS - 1); e += blockDim.x) {
        const int cc = e / (CH + KS - 1), j = e % (CH + KS - 1);
        int gi = i0 + j - KS / 2;
        gi = (gi % n + n) % n;
        xs[cc][j] = xsmp[(long long)cc * n + gi];
      }
      for (int e = threadIdx.x; e < 16 * CH; e += blockDim.x) {
        const int oo = e / CH, j = e % CH;
        gs[oo][j] = (o0 + oo < cout && i0 + j < n) ? gsmp[(long long)(o0 + oo) * n + i0 + j] : 0.f;
      }
      __syncthreads();
      if (c < cin) {
        const int len = min(CH, n - i0);
        for (int j = 0; j < len; ++j) {
          float xv[KS];
#pragma unroll
          for (int t = 0; t < KS; ++t) xv[t] = xs[c][j + t];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float gv = gs[os + a][j];
#pragma unroll
            for (int t = 0; t < KS; ++t) acc[a][t] = fmaf(gv, xv[t], acc[a][t]);
            if (c == 0) bacc[a] += gv;
          }
        }
      }
    }
  }
  if (c < cin) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int o = o0 + os + a;
      if (o >= cout) continue;
#pragma unroll
      for (int t = 0; t < KS; ++t) atomicAdd(dW + ((long long)o * cin + c) * KS + t, acc[a][t]);
      if (c == 0) atomicAdd(db + o, bacc[a]);
    }
  }
}

// g *= GELU'(pre)
__global__ void gelu_bwd_kernel(long long count, const float* pre, float* g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    g[i] *= gelu_grad_f(pre[i]);
}

// Features of a batch: x[s][0][i] = b/s_b, x[s][1][i] = dz0/s_z; target
// (dz_j - dz_0)/s_z (if sol is set).
__global__ void features_kernel(int n, int S, const int* idx, const double* rhs, const double* ctrl,
                                const double* sol, double sb, double sz, float* x, float* target) {
  const long long total = (long long)S * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), i = (int)(e % n);
    const long long src = (long long)(idx ? idx[s] : s) * n + i;
    x[((long long)s * 2) * n + i] = (float)(rhs[src] / sb);
    x[((long long)s * 2 + 1) * n + i] = (float)(ctrl[src] / sz);
    if (sol && target) target[e] = (float)((sol[src] - ctrl[src]) / sz);
  }
}

// MSE: loss += sum (out - target)^2 / m (FP64), g = 2 (out - target) / m.
__global__ void mse_kernel(long long m, const float* out, const float* target, float* g, double* loss) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const float d = out[i] - target[i];
    g[i] = 2.f * d / (float)m;
    s += (double)d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(loss, t / (double)m);
  }
}

// AdamW on the FP32 masters (bias-corrected, decoupled weight decay).
__global__ void adamw_kernel(long long count, float* theta, const float* grad, float* m, float* v, float lr, float wd,
                             float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    theta[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * theta[i]);
  }
}

// BF16 copies of a layer's weights: W [o][c][t] and its transpose-flip
// Wt [c][o][4 - t] (the data-gradient convolution).
__global__ void weights_bf16_kernel(int cout, int cin, const float* W, __nv_bfloat16* Wb, __nv_bfloat16* Wt) {
  const int total = cout * cin * KS;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int o = e / (cin * KS), c = (e / KS) % cin, t = e % KS;
    const __nv_bfloat16 b = __float2bfloat16_rn(W[e]);
    Wb[e] = b;
    Wt[((long long)c * cout + o) * KS + (KS - 1 - t)] = b;
  }
}

__global__ void guess_kernel(long long total, int n, const int* idx, const double* ctrl, const float* out, double sz,
                             double* dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / n;
    const long long src = (long long)(idx ? idx[s] : s) * n + (e % n);
    dst[src] = ctrl[src] + sz * (double)out[e];
  }
}

__global__ void sumsq_kernel(long long count, const double* v, double* acc) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    s += v[i] * v[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(acc, t);
  }
}

}  // namespace

// theta = eta * scale (He-scaled weights from standard-normal draws).
__global__ void he_init_kernel(long long count, const double* eta, float* theta, float scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    theta[i] = (float)eta[i] * scale;
}

struct eda_ws {
  int n = 0, H = 0, Bmax = 0;
  cudaStream_t st = nullptr;
  std::string err;
  int cin[4], cout_[4];
  long long woff[4], boff[4], nparam = 0;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *Wb = nullptr, *Wt = nullptr;  // per layer at woff
  // tensor-core tap tiles of the 64 -> 64 layers (forward, data gradient),
  // layer l at l * 5 * 64 * 64; tc: those layers run on the tensor cores
  __nv_bfloat16 *Tf = nullptr, *Tb = nullptr;
  bool tc = false;
  int* tout = nullptr;  // set by a tensor-core wait that gave up
  float* act[5] = {};                           // act[0] features, act[l] output of layer l
  float* pre[4] = {};                           // pre-activations of layers 1..3
  float* gbuf[2] = {};                          // gradient ping-pong (max channels)
  float* target = nullptr;
  double* dloss = nullptr;
  double* hpin = nullptr;
  int* didx = nullptr;
  double sb = 0.0, sz = 0.0;
  long long step = 0;
  std::vector<void*> allocs;
};

namespace {

int wfail(eda_ws* w, int code, const std::string& msg) {
  if (w) w->err = msg;
  return eda::fail(nullptr, code, msg);
}
#define WCU(w, ...)                                                                                \
  do {                                                                                             \
    cudaError_t e__ = (__VA_ARGS__);                                                               \
    if (e__ != cudaSuccess)                                                                        \
      return wfail((w), EDA_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__)); \
  } while (0)

template <typename T>
cudaError_t walloc(eda_ws* w, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
  if (e == cudaSuccess) w->allocs.push_back((void*)*p);
  return e;
}

// The tensor-core tap tiles of layer l (nullptr: the layer runs on CUDA cores).
const __nv_bfloat16* tile_f(const eda_ws* w, int l) {
  return w->tc && w->cin[l] == kTcCh && w->cout_[l] == kTcCh ? w->Tf + (long long)l * KS * kTcCh * kTcCh : nullptr;
}
const __nv_bfloat16* tile_b(const eda_ws* w, int l) {
  return w->tc && w->cin[l] == kTcCh && w->cout_[l] == kTcCh ? w->Tb + (long long)l * KS * kTcCh * kTcCh : nullptr;
}

int refresh_bf16(eda_ws* w) {
  for (int l = 0; l < 4; ++l) {
    eda::count_launch();
    weights_bf16_kernel<<<64, 256, 0, w->st>>>(w->cout_[l], w->cin[l], w->theta + w->woff[l], w->Wb + w->woff[l],
                                               w->Wt + w->woff[l]);
    if (tile_f(w, l) != nullptr) {
      eda::count_launch();
      weights_tile_kernel<<<80, 256, 0, w->st>>>(w->theta + w->woff[l], w->Tf + (long long)l * KS * kTcCh * kTcCh,
                                                 w->Tb + (long long)l * KS * kTcCh * kTcCh);
    }
  }
  WCU(w, cudaGetLastError());
  return EDA_OK;
}

// One convolution of S samples; tile != nullptr (a 64 -> 64 layer's tap
// tiles) runs it on the tensor cores.
int conv(eda_ws* w, int S, int cin, int cout, const float* x, const __nv_bfloat16* W, const __nv_bfloat16* tile,
         const float* b, float* pre, float* out, int act) {
  static bool attr = false;
  if (!attr) {
    WCU(w, cudaFuncSetAttribute(conv_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                MAXC * (TP + KS - 1) * 4 + MAXC * MAXC * KS * 2));
    WCU(w, cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
    attr = true;
  }
  eda::count_launch();
  if (tile != nullptr) {
    conv_tc_kernel<<<dim3(S, (w->n + kTcPos - 1) / kTcPos), 128, kTcSmem, w->st>>>(w->n, x, tile, b, pre, out, act,
                                                                                   w->tout);
  } else {
    const size_t smem =
        (size_t)cin * (TP + KS - 1) * sizeof(float) + (size_t)cout * cin * KS * sizeof(__nv_bfloat16);
    conv_fwd_kernel<<<dim3(S, (w->n + TP - 1) / TP), 256, smem, w->st>>>(w->n, cin, cout, x, W, b, pre, out, act);
  }
  WCU(w, cudaGetLastError());
  return EDA_OK;
}

// After the stream synchronised: EDA_ERR_TIMEOUT if a tensor-core wait gave up.
int check_tout(eda_ws* w) {
  if (!w->tc) return EDA_OK;
  int t = 0;
  WCU(w, cudaMemcpy(&t, w->tout, sizeof(int), cudaMemcpyDeviceToHost));
  if (t) {
    WCU(w, cudaMemset(w->tout, 0, sizeof(int)));
    return wfail(w, EDA_ERR_TIMEOUT, "warm start: a bounded wait for the tensor cores gave up");
  }
  return EDA_OK;
}

// Forward of S samples whose features are in act[0].
int forward(eda_ws* w, int S) {
  for (int l = 0; l < 4; ++l) {
    const int rc = conv(w, S, w->cin[l], w->cout_[l], w->act[l], w->Wb + w->woff[l], tile_f(w, l),
                        w->theta + w->boff[l], l < 3 ? w->pre[l] : nullptr, w->act[l + 1], l < 3 ? 1 : 0);
    if (rc) return rc;
  }
  return EDA_OK;
}

// Loss (into dloss) and gradients (into grad) of S samples; features and
// targets staged.
int forward_backward(eda_ws* w, int S) {
  int rc = forward(w, S);
  if (rc) return rc;
  const long long mm = (long long)S * w->n;
  WCU(w, cudaMemsetAsync(w->grad, 0, w->nparam * sizeof(float), w->st));
  eda::count_launch();
  mse_kernel<<<eda::grid_for(mm), 256, 0, w->st>>>(mm, w->act[4], w->target, w->gbuf[0], w->dloss);
  WCU(w, cudaGetLastError());
  int cur = 0;
  for (int l = 3; l >= 0; --l) {
    float* g = w->gbuf[cur];
    if (l < 3) {
      const long long cnt = (long long)S * w->cout_[l] * w->n;
      eda::count_launch();
      gelu_bwd_kernel<<<eda::grid_for(cnt), 256, 0, w->st>>>(cnt, w->pre[l], g);
      WCU(w, cudaGetLastError());
    }
    eda::count_launch();
    const int slices = S < 64 ? S : 64;
    conv_wgrad_kernel<<<dim3((w->cout_[l] + 15) / 16, slices), 256, 0, w->st>>>(
        w->n, S, w->cin[l], w->cout_[l], w->act[l], g, w->grad + w->woff[l], w->grad + w->boff[l]);
    WCU(w, cudaGetLastError());
    if (l > 0) {
      rc = conv(w, S, w->cout_[l], w->cin[l], g, w->Wt + w->woff[l], tile_b(w, l), nullptr, nullptr,
                w->gbuf[1 - cur], 0);
      if (rc) return rc;
      cur = 1 - cur;
    }
  }
  return EDA_OK;
}

}  // namespace

extern "C" {

EDA_API int eda_ws_create(int n, int hidden, int max_batch, void* stream, eda_ws** out) {
  if (!out) return eda::fail(nullptr, EDA_ERR_INVALID, "eda_ws_create: out is NULL");
  *out = nullptr;
  if (n < KS || hidden < 1 || hidden > MAXC || max_batch < 1)
    return eda::fail(nullptr, EDA_ERR_INVALID, "eda_ws_create: need n >= 5, 1 <= hidden <= 64, max_batch >= 1");
  eda_ws* w = new eda_ws();
  w->n = n;
  w->H = hidden;
  w->Bmax = max_batch;
  w->st = (cudaStream_t)stream;
  const int ci[4] = {2, hidden, hidden, hidden}, co[4] = {hidden, hidden, hidden, 1};
  long long o = 0;
  for (int l = 0; l < 4; ++l) {
    w->cin[l] = ci[l];
    w->cout_[l] = co[l];
    w->woff[l] = o;
    o += (long long)co[l] * ci[l] * KS;
    w->boff[l] = o;
    o += co[l];
  }
  w->nparam = o;
  const long long B = max_batch;
  bool ok = !walloc(w, &w->theta, o) && !walloc(w, &w->grad, o) && !walloc(w, &w->m, o) && !walloc(w, &w->v, o) &&
            !walloc(w, &w->Wb, o) && !walloc(w, &w->Wt, o) && !walloc(w, &w->act[0], B * 2 * n) &&
            !walloc(w, &w->target, B * n) && !walloc(w, &w->dloss, 1) && !walloc(w, &w->didx, B);
  for (int l = 0; l < 4 && ok; ++l) {
    ok = !walloc(w, &w->act[l + 1], B * co[l] * n);
    if (ok && l < 3) ok = !walloc(w, &w->pre[l], B * co[l] * n);
  }
  for (int i = 0; i < 2 && ok; ++i) ok = !walloc(w, &w->gbuf[i], B * (long long)hidden * n);
  // the 64 -> 64 layers on the tensor cores (EDA_WS_TC=0: CUDA cores)
  w->tc = hidden == kTcCh && eda::env_int("EDA_WS_TC", 1) != 0;
  if (ok && w->tc) {
    const size_t tiles = (size_t)4 * KS * kTcCh * kTcCh;
    ok = !walloc(w, &w->Tf, tiles) && !walloc(w, &w->Tb, tiles) && !walloc(w, &w->tout, 1);
    if (ok) ok = cudaMemset(w->tout, 0, sizeof(int)) == cudaSuccess;
  }
  if (ok) ok = cudaMallocHost((void**)&w->hpin, 2 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    eda_ws_destroy(w);
    return eda::fail(nullptr, EDA_ERR_CUDA, "eda_ws_create: out of memory");
  }
  cudaMemsetAsync(w->theta, 0, o * sizeof(float), w->st);
  cudaMemsetAsync(w->m, 0, o * sizeof(float), w->st);
  cudaMemsetAsync(w->v, 0, o * sizeof(float), w->st);
  *out = w;
  return EDA_OK;
}

EDA_API int eda_ws_destroy(eda_ws* w) {
  if (!w) return EDA_OK;
  if (w->st) cudaStreamSynchronize(w->st);
  for (void* p : w->allocs) cudaFree(p);
  if (w->hpin) cudaFreeHost(w->hpin);
  delete w;
  return EDA_OK;
}

EDA_API const char* eda_ws_last_error(const eda_ws* w) { return w ? w->err.c_str() : eda_last_error(nullptr); }

EDA_API long long eda_ws_num_params(const eda_ws* w) { return w ? w->nparam : 0; }

EDA_API int eda_ws_init(eda_ws* w, const double* draws) {
  if (!w || !draws) return wfail(w, EDA_ERR_INVALID, "eda_ws_init: invalid argument");
  const double* eta = draws;
  double* tmp = nullptr;
  if (!eda::is_device_ptr(draws)) {
    WCU(w, cudaMalloc((void**)&tmp, w->nparam * sizeof(double)));
    WCU(w, cudaMemcpyAsync(tmp, draws, w->nparam * sizeof(double), cudaMemcpyHostToDevice, w->st));
    eta = tmp;
  }
  for (int l = 0; l < 4; ++l) {
    const long long nwt = (long long)w->cout_[l] * w->cin[l] * KS;
    eda::count_launch();
    he_init_kernel<<<eda::grid_for(nwt), 256, 0, w->st>>>(nwt, eta + w->woff[l], w->theta + w->woff[l],
                                                          (float)std::sqrt(2.0 / (w->cin[l] * KS)));
    WCU(w, cudaGetLastError());
    WCU(w, cudaMemsetAsync(w->theta + w->boff[l], 0, w->cout_[l] * sizeof(float), w->st));
  }
  WCU(w, cudaMemsetAsync(w->m, 0, w->nparam * sizeof(float), w->st));
  WCU(w, cudaMemsetAsync(w->v, 0, w->nparam * sizeof(float), w->st));
  w->step = 0;
  const int rc = refresh_bf16(w);
  if (rc) return rc;
  WCU(w, cudaStreamSynchronize(w->st));
  if (tmp) cudaFree(tmp);
  return EDA_OK;
}

EDA_API int eda_ws_set_params(eda_ws* w, const float* params) {
  if (!w || !params) return wfail(w, EDA_ERR_INVALID, "eda_ws_set_params: invalid argument");
  WCU(w, cudaMemcpyAsync(w->theta, params, w->nparam * sizeof(float), cudaMemcpyDefault, w->st));
  WCU(w, cudaMemsetAsync(w->m, 0, w->nparam * sizeof(float), w->st));
  WCU(w, cudaMemsetAsync(w->v, 0, w->nparam * sizeof(float), w->st));
  w->step = 0;
  const int rc = refresh_bf16(w);
  if (rc) return rc;
  WCU(w, cudaStreamSynchronize(w->st));
  return EDA_OK;
}

EDA_API int eda_ws_get_params(eda_ws* w, float* params) {
  if (!w || !params) return wfail(w, EDA_ERR_INVALID, "eda_ws_get_params: invalid argument");
  WCU(w, cudaMemcpyAsync(params, w->theta, w->nparam * sizeof(float), cudaMemcpyDefault, w->st));
  WCU(w, cudaStreamSynchronize(w->st));
  return EDA_OK;
}

EDA_API int eda_ws_set_scales(eda_ws* w, double s_b, double s_z) {
  if (!w || !(s_b > 0.0) || !(s_z > 0.0)) return wfail(w, EDA_ERR_INVALID, "eda_ws_set_scales: scales must be > 0");
  w->sb = s_b;
  w->sz = s_z;
  return EDA_OK;
}

EDA_API int eda_ws_get_scales(const eda_ws* w, double* s_b, double* s_z) {
  if (!w || !s_b || !s_z) return eda::fail(nullptr, EDA_ERR_INVALID, "eda_ws_get_scales: invalid argument");
  *s_b = w->sb;
  *s_z = w->sz;
  return EDA_OK;
}

EDA_API int eda_ws_loss_grad(eda_ws* w, const double* rhs, const double* ctrl, const double* sol, int count,
                             double* loss_out, float* grad_out) {
  if (!w || !rhs || !ctrl || !sol || count < 1 || count > w->Bmax)
    return wfail(w, EDA_ERR_INVALID, "eda_ws_loss_grad: invalid argument (count must be in [1, max_batch])");
  if (!(w->sb > 0.0)) return wfail(w, EDA_ERR_STATE, "eda_ws_loss_grad: scales not set");
  const size_t bytes = (size_t)count * w->n * sizeof(double);
  double *dr = nullptr, *dc = nullptr, *ds = nullptr;
  WCU(w, cudaMallocAsync((void**)&dr, bytes, w->st));
  WCU(w, cudaMallocAsync((void**)&dc, bytes, w->st));
  WCU(w, cudaMallocAsync((void**)&ds, bytes, w->st));
  WCU(w, cudaMemcpyAsync(dr, rhs, bytes, cudaMemcpyDefault, w->st));
  WCU(w, cudaMemcpyAsync(dc, ctrl, bytes, cudaMemcpyDefault, w->st));
  WCU(w, cudaMemcpyAsync(ds, sol, bytes, cudaMemcpyDefault, w->st));
  eda::count_launch();
  features_kernel<<<eda::grid_for((long long)count * w->n), 256, 0, w->st>>>(w->n, count, nullptr, dr, dc, ds, w->sb,
                                                                              w->sz, w->act[0], w->target);
  WCU(w, cudaGetLastError());
  WCU(w, cudaMemsetAsync(w->dloss, 0, sizeof(double), w->st));
  int rc = refresh_bf16(w);
  if (rc) return rc;
  rc = forward_backward(w, count);
  if (rc) return rc;
  WCU(w, cudaMemcpyAsync(w->hpin, w->dloss, sizeof(double), cudaMemcpyDeviceToHost, w->st));
  if (grad_out) WCU(w, cudaMemcpyAsync(grad_out, w->grad, w->nparam * sizeof(float), cudaMemcpyDefault, w->st));
  WCU(w, cudaFreeAsync(dr, w->st));
  WCU(w, cudaFreeAsync(dc, w->st));
  WCU(w, cudaFreeAsync(ds, w->st));
  WCU(w, cudaStreamSynchronize(w->st));
  rc = check_tout(w);
  if (rc) return rc;
  if (loss_out) *loss_out = w->hpin[0];
  return EDA_OK;
}

EDA_API int eda_ws_train(eda_ws* w, const double* rhs, const double* ctrl, const double* sol, int count, int epochs,
                         int batch, double lr, double weight_decay, const int* order, double* loss_out) {
  if (!w || !rhs || !ctrl || !sol || count < 1 || epochs < 0 || batch < 1 || batch > w->Bmax || !(lr > 0.0))
    return wfail(w, EDA_ERR_INVALID, "eda_ws_train: invalid argument");
  const size_t bytes = (size_t)count * w->n * sizeof(double);
  // training data on the device (host inputs are staged once)
  double *dr = (double*)rhs, *dc = (double*)ctrl, *ds = (double*)sol;
  bool staged = false;
  if (!eda::is_device_ptr(rhs) || !eda::is_device_ptr(ctrl) || !eda::is_device_ptr(sol)) {
    staged = true;
    WCU(w, cudaMallocAsync((void**)&dr, bytes, w->st));
    WCU(w, cudaMallocAsync((void**)&dc, bytes, w->st));
    WCU(w, cudaMallocAsync((void**)&ds, bytes, w->st));
    WCU(w, cudaMemcpyAsync(dr, rhs, bytes, cudaMemcpyDefault, w->st));
    WCU(w, cudaMemcpyAsync(dc, ctrl, bytes, cudaMemcpyDefault, w->st));
    WCU(w, cudaMemcpyAsync(ds, sol, bytes, cudaMemcpyDefault, w->st));
  }
  if (!(w->sb > 0.0)) {
    // input scales: RMS of b and of dz_0 over the training set
    double* acc = nullptr;
    WCU(w, cudaMallocAsync((void**)&acc, 2 * sizeof(double), w->st));
    WCU(w, cudaMemsetAsync(acc, 0, 2 * sizeof(double), w->st));
    const long long cnt = (long long)count * w->n;
    eda::count_launch(2);
    sumsq_kernel<<<eda::grid_for(cnt), 256, 0, w->st>>>(cnt, dr, acc);
    sumsq_kernel<<<eda::grid_for(cnt), 256, 0, w->st>>>(cnt, dc, acc + 1);
    WCU(w, cudaGetLastError());
    WCU(w, cudaMemcpyAsync(w->hpin, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, w->st));
    WCU(w, cudaFreeAsync(acc, w->st));
    WCU(w, cudaStreamSynchronize(w->st));
    w->sb = std::sqrt(w->hpin[0] / cnt);
    w->sz = std::sqrt(w->hpin[1] / cnt);
    if (!(w->sb > 0.0) || !(w->sz > 0.0)) return wfail(w, EDA_ERR_NUMERIC, "eda_ws_train: zero training data");
  }
  int* dorder = nullptr;
  if (order) {
    WCU(w, cudaMallocAsync((void**)&dorder, (size_t)epochs * count * sizeof(int), w->st));
    WCU(w, cudaMemcpyAsync(dorder, order, (size_t)epochs * count * sizeof(int), cudaMemcpyDefault, w->st));
  }
  int rc = refresh_bf16(w);
  if (rc) return rc;
  const float b1 = 0.9f, b2 = 0.999f;
  std::vector<double> eloss(epochs, 0.0);
  for (int ep = 0; ep < epochs; ++ep) {
    WCU(w, cudaMemsetAsync(w->dloss, 0, sizeof(double), w->st));
    int nb = 0;
    for (int s0 = 0; s0 < count; s0 += batch) {
      const int S = (count - s0 < batch) ? count - s0 : batch;
      const int* idx = nullptr;
      if (dorder) {
        idx = dorder + (long long)ep * count + s0;
      }
      eda::count_launch();
      features_kernel<<<eda::grid_for((long long)S * w->n), 256, 0, w->st>>>(
          w->n, S, idx, idx ? dr : dr + (long long)s0 * w->n, idx ? dc : dc + (long long)s0 * w->n,
          idx ? ds : ds + (long long)s0 * w->n, w->sb, w->sz, w->act[0], w->target);
      WCU(w, cudaGetLastError());
      rc = forward_backward(w, S);
      if (rc) return rc;
      ++w->step;
      const float c1 = 1.f - std::pow(b1, (float)w->step), c2 = 1.f - std::pow(b2, (float)w->step);
      eda::count_launch();
      adamw_kernel<<<eda::grid_for(w->nparam), 256, 0, w->st>>>(w->nparam, w->theta, w->grad, w->m, w->v, (float)lr,
                                                                 (float)weight_decay, b1, b2, 1e-8f, c1, c2);
      WCU(w, cudaGetLastError());
      rc = refresh_bf16(w);
      if (rc) return rc;
      ++nb;
    }
    WCU(w, cudaMemcpyAsync(w->hpin, w->dloss, sizeof(double), cudaMemcpyDeviceToHost, w->st));
    WCU(w, cudaStreamSynchronize(w->st));
    eloss[ep] = w->hpin[0] / (nb > 0 ? nb : 1);
  }
  if (dorder) WCU(w, cudaFreeAsync(dorder, w->st));
  if (staged) {
    WCU(w, cudaFreeAsync(dr, w->st));
    WCU(w, cudaFreeAsync(dc, w->st));
    WCU(w, cudaFreeAsync(ds, w->st));
  }
  WCU(w, cudaStreamSynchronize(w->st));
  rc = check_tout(w);
  if (rc) return rc;
  if (loss_out) std::memcpy(loss_out, eloss.data(), epochs * sizeof(double));
  return EDA_OK;
}

EDA_API int eda_ws_infer(eda_ws* w, const double* rhs, const double* ctrl, int count, double* out) {
  if (!w || !rhs || !ctrl || !out || count < 0) return wfail(w, EDA_ERR_INVALID, "eda_ws_infer: invalid argument");
  if (!(w->sb > 0.0)) return wfail(w, EDA_ERR_STATE, "eda_ws_infer: the network has no input scales (train first)");
  if (count == 0) return EDA_OK;
  const size_t bytes = (size_t)count * w->n * sizeof(double);
  const double *dr = rhs, *dc = ctrl;
  double* dout = out;
  void *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
  if (!eda::is_device_ptr(rhs)) {
    WCU(w, cudaMallocAsync(&t1, bytes, w->st));
    WCU(w, cudaMemcpyAsync(t1, rhs, bytes, cudaMemcpyDefault, w->st));
    dr = (const double*)t1;
  }
  if (!eda::is_device_ptr(ctrl)) {
    WCU(w, cudaMallocAsync(&t2, bytes, w->st));
    WCU(w, cudaMemcpyAsync(t2, ctrl, bytes, cudaMemcpyDefault, w->st));
    dc = (const double*)t2;
  }
  const bool host_out = !eda::is_device_ptr(out);
  if (host_out) {
    WCU(w, cudaMallocAsync(&t3, bytes, w->st));
    dout = (double*)t3;
  }
  int rc = refresh_bf16(w);
  if (rc) return rc;
  for (int s0 = 0; s0 < count; s0 += w->Bmax) {
    const int S = (count - s0 < w->Bmax) ? count - s0 : w->Bmax;
    const long long o = (long long)s0 * w->n;
    eda::count_launch();
    features_kernel<<<eda::grid_for((long long)S * w->n), 256, 0, w->st>>>(w->n, S, nullptr, dr + o, dc + o, nullptr,
                                                                            w->sb, w->sz, w->act[0], nullptr);
    WCU(w, cudaGetLastError());
    rc = forward(w, S);
    if (rc) return rc;
    eda::count_launch();
    guess_kernel<<<eda::grid_for((long long)S * w->n), 256, 0, w->st>>>((long long)S * w->n, w->n, nullptr, dc + o,
                                                                         w->act[4], w->sz, dout + o);
    WCU(w, cudaGetLastError());
  }
  if (host_out) WCU(w, cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, w->st));
  if (t1) WCU(w, cudaFreeAsync(t1, w->st));
  if (t2) WCU(w, cudaFreeAsync(t2, w->st));
  if (t3) WCU(w, cudaFreeAsync(t3, w->st));
  if (host_out || w->tc) WCU(w, cudaStreamSynchronize(w->st));
  return check_tout(w);
}

}  // extern "C"
