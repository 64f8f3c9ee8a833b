// Batched application of the scaled spectral LMP P_theta and of its
// symmetric factor U_theta (Section 3.1, Eq. (lmp)) to every member's
// vector: Z = R + S diag(coef) S^T R, the two dense contractions of the PCG
// iteration (S: n x k orthonormal columns, R: n x M, k <= 80, M <= 257).
//
// Two implementations of the same two launches (projections W = S^T R over
// row chunks, then the expansion Z = R + S (coef o W)):
//  * CUDA cores (lmp_apply_cc) in FP64, or FP32 with the FP32 copy of S;
//  * tensor cores (lmp_apply_tc): tcgen05.mma kind::f16 with BF16 operands
//    and FP32 accumulators in tensor memory.  Each operand x is split as
//    x = hi + lo with hi = bf16(x), lo = bf16(x - hi) (16 significant bits
//    together), and each product is taken as hi.hi + hi.lo + lo.hi into one
//    accumulator (the dropped lo.lo term is 2^-16 below it).  Shared-memory
//    operands use the canonical K-major, no-swizzle layout (core matrices of
//    8 rows x 16 bytes).  The S operand of each row chunk is stored in global
//    memory already in that layout (split_bf16), so one bulk asynchronous
//    copy per part (cp.async.bulk, completion counted on an mbarrier) moves
//    it while the CTA's threads split the member vectors into the other
//    operand.  One thread issues the MMAs and commits to a second mbarrier;
//    every wait is bounded; the epilogue reads the accumulator with
//    tcgen05.ld.  One CTA per SM and member tile works through every
//    gridDim.x-th row chunk in a two-stage pipeline (the projections
//    accumulate in tensor memory across the CTA's chunks; the expansion
//    double-buffers its accumulator to overlap its MMAs and epilogue).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "eda_internal.h"
#include "lmp.h"
#include "tc.h"

namespace eda {
namespace {

using namespace tc;

constexpr int kRows = 128;  // rows of n per CTA (a row chunk)

// ----------------------------------------------------------------- CUDA cores
constexpr int kCcThreads = 256;
constexpr int kCcWarps = kCcThreads / 32;
constexpr int kSmRow = kRows + 1;  // padded shared row: lanes reading one row per mode do not collide

template <typename TS>
__device__ __forceinline__ void stage_chunk(const TS* S, int n, int k, int row0, int rows, TS* sm) {
  for (int idx = threadIdx.x; idx < k * kRows; idx += kCcThreads) {
    const int c = idx / kRows, i = idx - c * kRows;
    sm[c * kSmRow + i] = i < rows ? S[(long long)c * n + row0 + i] : TS(0);
  }
}

template <typename TS>
__global__ void __launch_bounds__(kCcThreads) lmp_proj_cc_kernel(int n, int k, const TS* S, int M, const double* R,
                                                                 const int* active, TS* W, int kpad) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TS* Ssm = reinterpret_cast<TS*>(smraw);
  TS* rsm = Ssm + (size_t)k * kSmRow;  // [warp][kRows]
  const int row0 = blockIdx.x * kRows;
  const int rows = min(kRows, n - row0);
  stage_chunk<TS>(S, n, k, row0, rows, Ssm);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int m = blockIdx.y * kCcWarps + wid;
  const bool live = m < M && (active == nullptr || active[m] != 0);
  TS* rw = rsm + wid * kRows;
  for (int i = lane; i < kRows; i += 32) rw[i] = (live && i < rows) ? (TS)R[(long long)m * n + row0 + i] : TS(0);
  __syncthreads();
  if (!live) return;
  for (int c = lane; c < k; c += 32) {
    const TS* sc = Ssm + c * kSmRow;
    TS s0 = 0, s1 = 0;
    for (int i = 0; i < kRows; i += 2) {
      s0 += sc[i] * rw[i];
      s1 += sc[i + 1] * rw[i + 1];
    }
    atomicAdd(&W[(long long)m * kpad + c], s0 + s1);
  }
}

template <typename TS>
__global__ void __launch_bounds__(kCcThreads) lmp_expand_cc_kernel(int n, int k, const TS* S, const double* coef,
                                                                   int M, const double* R, double* Z,
                                                                   const int* active, const TS* W, int kpad) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TS* Ssm = reinterpret_cast<TS*>(smraw);
  TS* csm = Ssm + (size_t)k * kSmRow;  // [warp][k]: coef o w of the warp's member
  const int row0 = blockIdx.x * kRows;
  const int rows = min(kRows, n - row0);
  stage_chunk<TS>(S, n, k, row0, rows, Ssm);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int m = blockIdx.y * kCcWarps + wid;
  const bool live = m < M && (active == nullptr || active[m] != 0);
  TS* cw = csm + wid * k;
  if (live)
    for (int c = lane; c < k; c += 32) cw[c] = (TS)(coef[c] * (double)W[(long long)m * kpad + c]);
  __syncthreads();
  if (!live) return;
  for (int i = lane; i < rows; i += 32) {
    TS s0 = 0, s1 = 0;
    int c = 0;
    for (; c + 2 <= k; c += 2) {
      s0 += Ssm[c * kSmRow + i] * cw[c];
      s1 += Ssm[(c + 1) * kSmRow + i] * cw[c + 1];
    }
    if (c < k) s0 += Ssm[c * kSmRow + i] * cw[c];
    const long long g = (long long)m * n + row0 + i;
    Z[g] = R[g] + (double)(s0 + s1);
  }
}

// --------------------------------------------------------------- tensor cores
// core-matrix rows of R each thread loads at once (a 96-member tile of a
// chunk is 6 per thread: one round of loads in flight)
constexpr int kStageRows = 6;
constexpr int kTcThreads = 256;  // eight warps: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31
// FP64 -> FP32 by truncating the significand to 24 bits, in integer
// arithmetic (GB300's FP64 pipe, which its conversions use, runs at 1/64 of
// the FP32 rate).  Magnitudes below the FP32 normal range give a signed
// zero, above it (and NaN) a signed infinity.  The split below keeps 16
// significant bits, so truncation instead of rounding at bit 24 is of no
// consequence.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const unsigned int sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned int)e << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
}

// FP32 -> FP64, exactly, in integer arithmetic (FP32 subnormals give a
// signed zero; infinities and NaN keep their class).
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  const unsigned int ed = e == 0xFFu ? 0x7FFu : e - 127u + 1023u;
  return __hiloint2double((int)(sign | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// 8 values -> the 16-byte core-matrix rows of their BF16 high and low parts:
// hi = bf16(x), lo = bf16(x - hi), in FP32 arithmetic (x - hi is exact there:
// x carries 24 significant bits and hi its leading 8).
template <typename T>
__device__ __forceinline__ void split8(const T (&x)[8], uint4* hi, uint4* lo) {
  __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    float xf;
    if constexpr (sizeof(T) == 8)
      xf = f64_to_f32_trunc(x[e]);
    else
      xf = x[e];
    h[e] = __float2bfloat16_rn(xf);
    l[e] = __float2bfloat16_rn(xf - __bfloat162float(h[e]));
  }
  *hi = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
  *lo = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
}

// Thread 0: the kg/2 K-steps of hi.hi + hi.lo + lo.hi into the accumulator
// at dt (accumulate: add to what it holds), committed to the mbarrier at
// mma.  Operands K-major with kg = K/8 core-matrix groups along K (lbo 128,
// sbo kg * 128).
__device__ __forceinline__ void mma_split3_issue(uint32_t dt, const unsigned char* Ahi, const unsigned char* Alo,
                                                 const unsigned char* Bhi, const unsigned char* Blo, int kg, int nd,
                                                 bool accumulate, uint32_t mma) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t id = idesc_bf16(nd);
  const uint32_t sbo = (uint32_t)kg * 128u;
  for (int ks = 0; ks < kg / 2; ++ks) {
    const uint32_t o = (uint32_t)ks * 256u;  // two core matrices along K per step of 16
    const uint64_t ah = kmajor_desc(smem_u32(Ahi) + o, 128u, sbo);
    const uint64_t al = kmajor_desc(smem_u32(Alo) + o, 128u, sbo);
    const uint64_t bh = kmajor_desc(smem_u32(Bhi) + o, 128u, sbo);
    const uint64_t bl = kmajor_desc(smem_u32(Blo) + o, 128u, sbo);
    mma_bf16(dt, ah, bh, id, (accumulate || ks > 0) ? 1u : 0u);
    mma_bf16(dt, ah, bl, id, 1u);
    mma_bf16(dt, al, bh, id, 1u);
  }
  mma_commit(mma);
}

// Shared memory of the two kernels: two stages of A hi | A lo (bulk-copied
// S tiles) and, for the projections, B hi | B lo (split R tiles); then the
// mbarriers (bulk copies and MMAs of each stage), the TMEM slot and the
// abort flag.
struct TcStage {
  unsigned char *Ahi, *Alo, *Bhi, *Blo;
};

struct TcPipe {
  TcStage st[2];
  uint32_t tma[2], mma[2];
  uint32_t* slot;
  int* abort;
};

__device__ __forceinline__ TcPipe tc_pipe(unsigned char* sm, uint32_t a_bytes, uint32_t b_bytes) {
  TcPipe p;
  unsigned char* c = sm;
  for (int s = 0; s < 2; ++s) {
    p.st[s].Ahi = c;
    p.st[s].Alo = c + a_bytes;
    p.st[s].Bhi = c + 2 * a_bytes;
    p.st[s].Blo = c + 2 * a_bytes + b_bytes;
    c += 2 * (a_bytes + b_bytes);
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(c);
  for (int s = 0; s < 2; ++s) {
    p.tma[s] = smem_u32(bars + s);
    p.mma[s] = smem_u32(bars + 2 + s);
  }
  p.slot = reinterpret_cast<uint32_t*>(bars + 4);
  p.abort = reinterpret_cast<int*>(p.slot + 1);
  return p;
}

// Thread 0: the four mbarriers (count 1) and the abort flag.
__device__ __forceinline__ void tc_pipe_init(const TcPipe& p) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(p.tma[s]) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(p.mma[s]) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *p.abort = 0;
  }
}

// Thread 0: the bulk copies of the two parts of A (a_bytes each) into stage s.
__device__ __forceinline__ void tc_load_a(const TcPipe& p, int s, const __nv_bfloat16* hi, const __nv_bfloat16* lo,
                                          uint32_t a_bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(p.tma[s]), "r"(2u * a_bytes)
               : "memory");
  bulk_g2s(smem_u32(p.st[s].Ahi), hi, a_bytes, p.tma[s]);
  bulk_g2s(smem_u32(p.st[s].Alo), lo, a_bytes, p.tma[s]);
}

// Thread 0, once stage s's bulk copies (use u of the stage) have landed:
// the MMAs of the stage into dt, committed to the stage's MMA barrier.  If
// the wait gives up (or an earlier one did), the CTA is marked aborted and
// thread 0 arrives on the barrier itself, so that every later wait on it
// still ends.
__device__ __forceinline__ void tc_mma_stage(const TcPipe& p, int s, int u, uint32_t dt, int kg, int nd,
                                             bool accumulate) {
  if (*p.abort == 0 && !mbar_wait(p.tma[s], (uint32_t)(u & 1))) *p.abort = 1;
  if (*p.abort == 0)
    mma_split3_issue(dt, p.st[s].Ahi, p.st[s].Alo, p.st[s].Bhi, p.st[s].Blo, kg, nd, accumulate, p.mma[s]);
  else
    mbar_arrive(p.mma[s]);
}

// Every thread: waits (bounded) for use u of stage s's MMA barrier; true in
// every thread when it completed in all of them and nothing aborted.  A
// barrier completes in use order, so parity u & 1 names use u.
__device__ __forceinline__ bool tc_wait_mma(const TcPipe& p, int s, int u) {
  const bool ok = mbar_wait(p.mma[s], (uint32_t)(u & 1));
  return __syncthreads_and((ok && *p.abort == 0) ? 1 : 0) != 0;
}

// After a wait gave up: *timeout set, and every stage's outstanding bulk
// copies and MMAs given a second bounded wait before tensor memory is freed.
__device__ __forceinline__ void tc_drain(const TcPipe& p, int uses0, int uses1, int* timeout) {
  if (threadIdx.x == 0 && timeout != nullptr) atomicExch(timeout, 1);
  const int uses[2] = {uses0, uses1};
  for (int s = 0; s < 2; ++s)
    if (uses[s] > 0) {
      mbar_wait(p.tma[s], (uint32_t)((uses[s] - 1) & 1));
      mbar_wait(p.mma[s], (uint32_t)((uses[s] - 1) & 1));
    }
  __syncthreads();
}

// Projections W[m][c] += sum_i S[c][i] R[m][i] over the CTA's row chunks q =
// blockIdx.x, blockIdx.x + gridDim.x, ...: D (128 modes x mt members) =
// A (modes x rows) B (rows x members) accumulates in tensor memory across
// the chunks (K = 128 rows each) and is added into W once per CTA.  A is the
// chunk's tile of the projection copies (modes >= k zero), bulk-copied; B is
// R of the tile's members, split on the fly, six core-matrix rows in flight
// per thread (16-byte loads where R's rows allow them).  Two stages: chunk
// i + 1 is staged while the MMAs of chunk i run.
__global__ void __launch_bounds__(kTcThreads) lmp_proj_tc_kernel(int n, int k, const __nv_bfloat16* Ph,
                                                                 const __nv_bfloat16* Pl, int M, int mt, int chunks,
                                                                 const double* R, int vec, const int* active,
                                                                 float* W, int kt, int* timeout) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int KG = kRows / 8;  // 16 groups of 8 rows along K
  constexpr uint32_t kA = 128u * kRows * 2u;
  const TcPipe p = tc_pipe(sm, kA, (uint32_t)mt * kRows * 2u);
  const int m0 = blockIdx.y * mt;
  const int nq = (chunks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int ncols = tmem_cols(mt);
  tc_pipe_init(p);
  const uint32_t tbase = tmem_alloc(p.slot, ncols);  // includes the block barrier
  const int items = mt * KG;
  bool ok = true;
  int uses[2] = {0, 0};
  for (int i = 0; i < nq && ok; ++i) {
    const int s = i & 1;
    const int q = (int)blockIdx.x + i * (int)gridDim.x;
    const int row0 = q * kRows;
    const int rows = min(kRows, n - row0);
    // the stage's buffers were read by the MMAs of chunk i - 2
    if (i >= 2) ok = tc_wait_mma(p, s, uses[s] - 1);
    if (!ok) break;
    if (threadIdx.x == 0)
      tc_load_a(p, s, Ph + (long long)q * 128 * kRows, Pl + (long long)q * 128 * kRows, kA);
    for (int base = threadIdx.x; base < items; base += kStageRows * kTcThreads) {
      double x[kStageRows][8];
#pragma unroll
      for (int u = 0; u < kStageRows; ++u) {
        const int idx = base + u * kTcThreads;
        const int j = idx / KG, kb = idx - j * KG;
        const int m = m0 + j;
        const int i0 = 8 * kb;
        const bool live = idx < items && m < M && (active == nullptr || active[m] != 0);
        const double* src = R + (long long)m * n + row0 + i0;
        if (live && vec && i0 + 8 <= rows) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const double2 v = reinterpret_cast<const double2*>(src)[e];
            x[u][2 * e] = v.x;
            x[u][2 * e + 1] = v.y;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) x[u][e] = (live && i0 + e < rows) ? src[e] : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < kStageRows; ++u) {
        const int idx = base + u * kTcThreads;
        if (idx < items) {
          const int j = idx / KG, kb = idx - j * KG;
          uint4 h, l;
          split8<double>(x[u], &h, &l);
          *reinterpret_cast<uint4*>(p.st[s].Bhi + kmaj_off(j, kb, KG)) = h;
          *reinterpret_cast<uint4*>(p.st[s].Blo + kmaj_off(j, kb, KG)) = l;
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) tc_mma_stage(p, s, uses[s], tbase, KG, mt, i > 0);
    ++uses[s];
  }
  // the last commit follows every earlier MMA of this thread
  if (ok) {
    const int sl = (nq - 1) & 1;
    ok = tc_wait_mma(p, sl, uses[sl] - 1);
  }
  if (!ok) tc_drain(p, uses[0], uses[1], timeout);
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) ... (modes), column blocks of 16
    // members alternating between the two warps of a lane quarter
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3;
    const int mo = 32 * qd + lane;
    for (int c0 = 16 * (w >> 2); c0 < mt; c0 += 32) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)c0, v);
      if (mo < k) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int m = m0 + c0 + e;
          if (m < M && (active == nullptr || active[m] != 0)) atomicAdd(&W[(long long)m * kt + mo], v[e]);
        }
      }
    }
  }
  tmem_free(tbase, ncols);
}

// Expansion Z[m][i] = R[m][i] + sum_c S[c][i] coef[c] W[m][c] over the CTA's
// row chunks: D (128 rows x mt members) = A (128 rows x kt modes) B (kt
// modes x members).  B, coef o w of the tile's members split on the fly, is
// the same for every chunk and staged once; A, the chunk's tile of the
// expansion copies, is bulk-copied two chunks ahead into two stages, and D
// is double-buffered in tensor memory, so the copy of chunk i + 2 and the
// MMAs of chunk i + 1 run while the epilogue of chunk i reads R and writes Z.
__global__ void __launch_bounds__(kTcThreads) lmp_expand_tc_kernel(int n, int k, const __nv_bfloat16* Eh,
                                                                   const __nv_bfloat16* El, const double* coef,
                                                                   int M, int mt, int chunks, const double* R,
                                                                   double* Z, const int* active, const float* W,
                                                                   int kt, int* timeout) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int KG = kt / 8;
  const uint32_t kA = 128u * (uint32_t)kt * 2u;
  const uint32_t kB = (uint32_t)mt * (uint32_t)kt * 2u;
  // one B for both stages: stage 1 reads stage 0's B buffers
  TcPipe p = tc_pipe(sm, kA, kB);
  p.st[1].Bhi = p.st[0].Bhi;
  p.st[1].Blo = p.st[0].Blo;
  const int m0 = blockIdx.y * mt;
  const int nq = (chunks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int ncols = tmem_cols(2 * mt);  // two accumulators of mt columns
  auto chunk_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };
  int uses[2] = {0, 0};  // bulk copies (and MMAs) started per stage
  tc_pipe_init(p);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 && i < nq; ++i)
      tc_load_a(p, i, Eh + (long long)chunk_of(i) * 128 * kt, El + (long long)chunk_of(i) * 128 * kt, kA);
  }
  for (int i = 0; i < 2 && i < nq; ++i) ++uses[i];
  for (int idx = threadIdx.x; idx < mt * KG; idx += kTcThreads) {
    const int j = idx / KG, kb = idx - j * KG;
    const int m = m0 + j;
    const bool live = m < M && (active == nullptr || active[m] != 0);
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = 8 * kb + e;
      x[e] = (live && c < k) ? f64_to_f32_trunc(coef[c]) * W[(long long)m * kt + c] : 0.0f;
    }
    uint4 h, l;
    split8<float>(x, &h, &l);
    *reinterpret_cast<uint4*>(p.st[0].Bhi + kmaj_off(j, kb, KG)) = h;
    *reinterpret_cast<uint4*>(p.st[0].Blo + kmaj_off(j, kb, KG)) = l;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint32_t tbase = tmem_alloc(p.slot, ncols);  // includes the block barrier
  if (threadIdx.x == 0) tc_mma_stage(p, 0, 0, tbase, KG, mt, false);
  bool ok = true;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = w & 3;
  const int il = 32 * qd + lane;  // TMEM lane = accumulator row = row of the chunk
  for (int i = 0; i < nq && ok; ++i) {
    const int s = i & 1, s1 = s ^ 1;
    // chunk i's MMAs (use i / 2 of stage s) are done: its accumulator is
    // ready and stage s's A is free
    ok = tc_wait_mma(p, s, i >> 1);
    if (!ok) break;
    if (threadIdx.x == 0) {
      if (i + 2 < nq)
        tc_load_a(p, s, Eh + (long long)chunk_of(i + 2) * 128 * kt, El + (long long)chunk_of(i + 2) * 128 * kt,
                  kA);
      // chunk i + 1 into the other accumulator (read by the epilogue of
      // chunk i - 1, which ended at the last block barrier)
      if (i + 1 < nq) tc_mma_stage(p, s1, (i + 1) >> 1, tbase + (uint32_t)(s1 * mt), KG, mt, false);
    }
    if (i + 2 < nq) ++uses[s];
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row0 = chunk_of(i) * kRows;
    const int rows = min(kRows, n - row0);
    // the warp's column groups of 16 (groups w / 4, w / 4 + 2, w / 4 + 4 of
    // the at most six): every load of R first, then the stores (Z may alias
    // R: each element is read before this thread writes it)
    float v[3][16];
    double rv[3][16];
#pragma unroll
    for (int gg = 0; gg < 3; ++gg) {
      const int c0 = 16 * ((w >> 2) + 2 * gg);
      if (c0 < mt) tmem_ld16(tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(s * mt + c0), v[gg]);
    }
#pragma unroll
    for (int gg = 0; gg < 3; ++gg) {
      const int c0 = 16 * ((w >> 2) + 2 * gg);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int m = m0 + c0 + e;
        const bool on = c0 < mt && il < rows && m < M && (active == nullptr || active[m] != 0);
        rv[gg][e] = on ? R[(long long)m * n + row0 + il] : 0.0;
      }
    }
#pragma unroll
    for (int gg = 0; gg < 3; ++gg) {
      const int c0 = 16 * ((w >> 2) + 2 * gg);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int m = m0 + c0 + e;
        if (c0 < mt && il < rows && m < M && (active == nullptr || active[m] != 0))
          Z[(long long)m * n + row0 + il] = rv[gg][e] + f32_to_f64_exact(v[gg][e]);
      }
    }
    // accumulator s is read: the MMAs of chunk i + 2 may write it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok) tc_drain(p, uses[0], uses[1], timeout);
  tmem_free(tbase, ncols);
}

// The tiled BF16 copies of S [k x n] (column-major FP64): for every chunk of
// 128 rows, the projection operand (128 modes x 128 rows, K-major along the
// rows) and the expansion operand (128 rows x kt modes, K-major along the
// modes), each as high and low parts in the core-matrix layout shared memory
// takes; zero outside k x n.
__global__ void split_bf16_kernel(int n, int nS, int k, int kt, const double* S, __nv_bfloat16* Ph,
                                  __nv_bfloat16* Pl, __nv_bfloat16* Eh, __nv_bfloat16* El) {
  const long long total = 128LL * nS;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / nS), gi = (int)(e - (long long)c * nS);
    const double x = (c < k && gi < n) ? S[(long long)c * n + gi] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    const __nv_bfloat16 l = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
    const int q = gi / kRows, r = gi - q * kRows;
    const long long pe = (long long)q * 128 * kRows + (kmaj_off(c, r >> 3, kRows / 8) >> 1) + (r & 7);
    Ph[pe] = h;
    Pl[pe] = l;
    if (c < kt) {
      const long long ee = (long long)q * 128 * kt + (kmaj_off(r, c >> 3, kt >> 3) >> 1) + (c & 7);
      Eh[ee] = h;
      El[ee] = l;
    }
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

int lmp_tc_kt(int k) { return ((k + 15) / 16) * 16; }
int lmp_tc_ns(int n) { return ((n + kRows - 1) / kRows) * kRows; }
size_t lmp_tc_elems(int n, int k) {
  const size_t nS = (size_t)lmp_tc_ns(n);
  return 2 * nS * 128 + 2 * nS * (size_t)lmp_tc_kt(k);
}

template <typename TS>
cudaError_t lmp_apply_cc(int n, int k, const TS* S, const double* coef, int M, const double* R, double* Z,
                         const int* active, TS* W, int kpad, cudaStream_t s) {
  if (M <= 0 || n <= 0) return cudaSuccess;
  if (k <= 0) {
    if (Z == R) return cudaSuccess;
    return cudaMemcpyAsync(Z, R, (size_t)M * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaError_t e = cudaMemsetAsync(W, 0, (size_t)M * kpad * sizeof(TS), s);
  if (e != cudaSuccess) return e;
  const dim3 grid((n + kRows - 1) / kRows, (M + kCcWarps - 1) / kCcWarps);
  const size_t sm1 = ((size_t)k * kSmRow + (size_t)kCcWarps * kRows) * sizeof(TS);
  const size_t sm2 = ((size_t)k * kSmRow + (size_t)kCcWarps * k) * sizeof(TS);
  if ((e = set_smem(lmp_proj_cc_kernel<TS>, sm1)) != cudaSuccess) return e;
  if ((e = set_smem(lmp_expand_cc_kernel<TS>, sm2)) != cudaSuccess) return e;
  count_launch(2);
  lmp_proj_cc_kernel<TS><<<grid, kCcThreads, sm1, s>>>(n, k, S, M, R, active, W, kpad);
  lmp_expand_cc_kernel<TS><<<grid, kCcThreads, sm2, s>>>(n, k, S, coef, M, R, Z, active, W, kpad);
  return cudaGetLastError();
}

cudaError_t lmp_apply_tc(int n, int k, const __nv_bfloat16* tiles, const double* coef, int M, const double* R,
                         double* Z, const int* active, float* W, int* timeout, cudaStream_t s) {
  if (M <= 0 || n <= 0) return cudaSuccess;
  const int kt = lmp_tc_kt(k), nS = lmp_tc_ns(n);
  if (k <= 0 || kt > 128) return cudaErrorInvalidValue;
  const __nv_bfloat16* Ph = tiles;
  const __nv_bfloat16* Pl = Ph + (size_t)nS * 128;
  const __nv_bfloat16* Eh = Pl + (size_t)nS * 128;
  const __nv_bfloat16* El = Eh + (size_t)nS * kt;
  const int Mp = ((M + 15) / 16) * 16;
  cudaError_t e = cudaMemsetAsync(W, 0, (size_t)Mp * kt * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const int chunks = nS / kRows;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      (void)cudaGetLastError();
      sms = 152;
    }
  }
  // member tiles: multiples of 16 and at most 96 members (two pipeline
  // stages of the projection's operands then fit shared memory); more tiles
  // where the row chunks alone would leave SMs idle
  int mtiles = std::max((Mp + 95) / 96, std::min(Mp / 16, (sms + chunks - 1) / chunks));
  const int mt = (((Mp + mtiles - 1) / mtiles + 15) / 16) * 16;
  mtiles = (Mp + mt - 1) / mt;
  // one CTA per SM (the stages take most of its shared memory), each
  // working through every gridDim.x-th row chunk
  const int nblk = std::max(1, std::min(chunks, sms / mtiles));
  // 16-byte loads of R where every row starts on a 16-byte boundary
  const int vec = ((reinterpret_cast<uintptr_t>(R) & 15u) == 0 && (n & 1) == 0) ? 1 : 0;
  const size_t aP = (size_t)128 * kRows * 2, bP = (size_t)mt * kRows * 2;
  const size_t aE = (size_t)128 * kt * 2, bE = (size_t)mt * kt * 2;
  const size_t sm1 = 4 * (aP + bP) + 48, sm2 = 4 * (aE + bE) + 48;
  if ((e = set_smem(lmp_proj_tc_kernel, sm1)) != cudaSuccess) return e;
  if ((e = set_smem(lmp_expand_tc_kernel, sm2)) != cudaSuccess) return e;
  const dim3 grid((unsigned)nblk, (unsigned)mtiles);
  count_launch(2);
  lmp_proj_tc_kernel<<<grid, kTcThreads, sm1, s>>>(n, k, Ph, Pl, M, mt, chunks, R, vec, active, W, kt, timeout);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  lmp_expand_tc_kernel<<<grid, kTcThreads, sm2, s>>>(n, k, Eh, El, coef, M, mt, chunks, R, Z, active, W, kt,
                                                     timeout);
  return cudaGetLastError();
}

cudaError_t split_bf16(int n, int k, const double* S, __nv_bfloat16* tiles, cudaStream_t s) {
  const int kt = lmp_tc_kt(k), nS = lmp_tc_ns(n);
  __nv_bfloat16* Ph = tiles;
  __nv_bfloat16* Pl = Ph + (size_t)nS * 128;
  __nv_bfloat16* Eh = Pl + (size_t)nS * 128;
  __nv_bfloat16* El = Eh + (size_t)nS * kt;
  count_launch();
  long long blocks = (128LL * nS + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  split_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, nS, k, kt, S, Ph, Pl, Eh, El);
  return cudaGetLastError();
}

template cudaError_t lmp_apply_cc<double>(int, int, const double*, const double*, int, const double*, double*,
                                          const int*, double*, int, cudaStream_t);
template cudaError_t lmp_apply_cc<float>(int, int, const float*, const double*, int, const double*, double*,
                                         const int*, float*, int, cudaStream_t);

}  // namespace eda
