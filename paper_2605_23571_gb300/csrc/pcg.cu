// Row-chunk kernels of the batched PCG iteration (see pcg.h).
#include <vector>

#include "eda_internal.h"
#include "pcg.h"

namespace eda {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The row chunk and problem of this CTA.
__device__ __forceinline__ void grid_task(const PcgGrid& G, PcgTask* tk, PcgProb* P) {
  if (G.single) {
    *P = G.one;
    const int r0 = (int)blockIdx.x * kPcgRows;
    *tk = PcgTask{0, r0, min(kPcgRows, G.one.n - r0), blockIdx.x == 0 ? 1 : 0};
  } else {
    *tk = G.tasks[blockIdx.x];
    *P = G.probs[tk->prob];
  }
}

// 16-byte vectors of the LMP arithmetic type: VW values per load.
template <typename TS>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int VW = 4;
  __device__ static float dot(const float4& a, const float4& b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int VW = 2;
  __device__ static double dot(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }
};

// Stride (in values) of shared-memory rows read with 16-byte loads by
// consecutive lanes: a multiple of the vector width whose eight consecutive
// rows start in eight different 4-bank groups (4 mod 8 floats, 2 mod 4
// doubles), at least len.
template <typename TS>
__host__ __device__ __forceinline__ int vec_stride(int len) {
  constexpr int VW = 16 / (int)sizeof(TS);
  int st = ((len + VW - 1) / VW) * VW;
  while ((st / VW) % 2 == 0) st += VW;
  return st;
}

static_assert(kPcgRows == 128, "stage_S indexes full chunks by shift and mask");

// Stages rows [row0, row0 + rows) of the k columns of S (column c at
// S + c * n) into shared memory, sm[c * cs + i * rs] = S[c * n + row0 + i],
// with 16 loads in flight per thread before their stores.
template <typename TS>
__device__ __forceinline__ void stage_S(const TS* S, int n, int k, int row0, int rows, TS* sm, int cs, int rs) {
  constexpr int U = 16;
  const int total = k * rows;
  const bool full = rows == kPcgRows;  // a power of two: shift and mask
  for (int base = 0; base < total; base += U * kThreads) {
    TS v[U];
    int dst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + (int)threadIdx.x + u * kThreads;
      dst[u] = -1;
      if (idx < total) {
        const int c = full ? (idx >> 7) : idx / rows;
        const int i = idx - c * rows;
        v[u] = S[(long long)c * n + row0 + i];
        dst[u] = c * cs + i * rs;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (dst[u] >= 0) sm[dst[u]] = v[u];
  }
}

// Rows of a row chunk per lane (kPcgRows / 32): the warp of a member keeps
// its rows of the PCG vectors in registers, loaded before the CTA stages S so
// that both sets of global loads are in flight together.
constexpr int kRowsPerLane = kPcgRows / 32;
// LMP modes per lane in the precond launch: k <= 80 modes (the library's
// limit on ell) pad to at most 96 = 3 x 32 values
constexpr int kCwPerLane = 3;
static_assert(32 * kCwPerLane >= 84 && 32 * kCwPerLane >= 82, "padded k of 80 LMP modes fits");

template <typename TS>
__global__ void __launch_bounds__(kThreads) pcg2_update_kernel(const PcgGrid G, int kmax,
                                                               const double* p, const double* q, double* x,
                                                               double* r, PcgScalars* sc, PcgAcc* acc, int* active,
                                                               TS* Wk, int par, int update, int use_lmp,
                                                               int* nactive) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using V = typename Vec16<TS>::type;
  constexpr int VW = Vec16<TS>::VW;
  constexpr int R = kRowsPerLane;
  const int RBP = vec_stride<TS>(kPcgRows);  // S chunk [c][RBP]: lane c reads column c
  PcgTask tk;
  PcgProb P;
  grid_task(G, &tk, &P);
  const int k = use_lmp ? P.k : 0;
  const int rows_v = ((tk.rows + VW - 1) / VW) * VW;  // rows padded to whole vectors
  TS* Ssm = reinterpret_cast<TS*>(smraw);
  TS* rsm = Ssm + (size_t)kmax * RBP;  // [kWarps][kPcgRows]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // this warp's member (one member per warp) and its rows, loaded first
  const int m = blockIdx.y * kWarps + wid;
  const int item = P.item0 + m;
  // a handle's solve (one problem, at most a few hundred members) issues the
  // loads without waiting for the member's active flag (their addresses are
  // valid for every member; inactive members drop them); the group path,
  // whose thousands of members are mostly inactive late in a solve, tests
  // the flag first so that it does not stream their rows
  const bool live_flag = m < P.M && active[item] != 0;
  const bool mine = G.single ? m < P.M : live_flag;
  const bool live = live_flag;
  const long long off = P.off0 + (long long)m * P.n + tk.row0;
  double pv[R], qv[R], xv[R], rv[R], bv[R];
  double pq = 0.0, rzp = 0.0;
  const bool rec = update && P.jhist != nullptr;  // cost record: b is read too
  if (mine) {
    if (update) {
      pq = acc[item].pq;
      rzp = acc[item].rz[par];
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = lane + 32 * j;
      if (i < tk.rows) {
        rv[j] = r[off + i];
        if (update) {
          pv[j] = p[off + i];
          qv[j] = q[off + i];
          xv[j] = x[off + i];
        }
        if (rec) bv[j] = P.b[off + i];
      }
    }
  }
  const TS* S = static_cast<const TS*>(P.S);
  stage_S<TS>(S, P.n, k, tk.row0, tk.rows, Ssm, RBP, 1);
  for (int idx = threadIdx.x; idx < k * (rows_v - tk.rows); idx += kThreads) {
    const int c = idx / (rows_v - tk.rows);
    Ssm[c * RBP + tk.rows + (idx - c * (rows_v - tk.rows))] = TS(0);
  }
  // slot par^1 collects r.z in the precond launch that follows
  if (update && tk.first && blockIdx.y == 0)
    for (int mm = threadIdx.x; mm < P.M; mm += kThreads) acc[P.item0 + mm].rz[par ^ 1] = 0.0;
  __syncthreads();
  if (!live) return;
  TS* rw = rsm + wid * kPcgRows;
  if (update) {
    if (!(pq > 0.0)) {  // breakdown (or NaN): every CTA skips the member
      if (tk.first && lane == 0) {
        sc[item].status = isfinite(pq) ? EDA_BREAKDOWN : EDA_NAN;
        active[item] = 0;
        atomicSub(nactive, 1);
      }
      return;
    }
    const double alpha = rzp / pq;
    double rr = 0.0, xx = 0.0, jx = 0.0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = lane + 32 * j;
      if (i < tk.rows) {
        const double xn = xv[j] + alpha * pv[j];
        x[off + i] = xn;
        const double rn = rv[j] - alpha * qv[j];
        r[off + i] = rn;
        rr += rn * rn;
        xx += xn * xn;
        if (rec) jx += xn * (bv[j] + rn);
        rw[i] = (TS)rn;
      }
    }
    rr = warp_sum(rr);
    if (lane == 0) atomicAdd(&acc[item].rr, rr);
    if (P.etol > 0.0) {
      xx = warp_sum(xx);
      if (lane == 0) atomicAdd(&acc[item].xx, xx);
    }
    if (rec) {
      jx = warp_sum(jx);
      if (lane == 0) atomicAdd(&acc[item].jx, jx);
    }
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = lane + 32 * j;
      if (i < tk.rows) rw[i] = (TS)rv[j];
    }
  }
  if (lane < rows_v - tk.rows) rw[tk.rows + lane] = TS(0);
  __syncwarp();
  for (int c = lane; c < k; c += 32) {
    const V* Sc = reinterpret_cast<const V*>(Ssm + c * RBP);
    const V* rvv = reinterpret_cast<const V*>(rw);
    TS s0 = 0, s1 = 0;
    int i = 0;
    for (; i + 2 <= rows_v / VW; i += 2) {
      s0 += Vec16<TS>::dot(Sc[i], rvv[i]);
      s1 += Vec16<TS>::dot(Sc[i + 1], rvv[i + 1]);
    }
    if (i < rows_v / VW) s0 += Vec16<TS>::dot(Sc[i], rvv[i]);
    atomicAdd(&Wk[(long long)item * kmax + c], s0 + s1);
  }
}

template <typename TS>
__global__ void __launch_bounds__(kThreads) pcg2_precond_kernel(const PcgGrid G, int kmax,
                                                                const double* r, double* z, double* p,
                                                                PcgScalars* sc, PcgAcc* acc, int* active,
                                                                const TS* Wk, int par, double tol, int maxit,
                                                                int fixed, int use_lmp, int init, int* nactive,
                                                                const double* zpre) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using V = typename Vec16<TS>::type;
  constexpr int VW = Vec16<TS>::VW;
  constexpr int R = kRowsPerLane;
  PcgTask tk;
  PcgProb P;
  grid_task(G, &tk, &P);
  const int k = use_lmp ? P.k : 0;
  const int KP = vec_stride<TS>(k);               // row stride, zero beyond k
  const int KW = vec_stride<TS>(kmax > 0 ? kmax : 1);
  TS* Ssm = reinterpret_cast<TS*>(smraw);        // [row][KP]: lane = row reads a row
  TS* wsm = Ssm + (size_t)kPcgRows * KW;         // [kWarps][KW]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // this warp's member, its rows of r, its stopping-test inputs and its
  // scaled projections, loaded before the CTA stages S
  const int m = blockIdx.y * kWarps + wid;
  const int item = P.item0 + m;
  const bool live_flag = m < P.M && active[item] != 0;  // loads as in the update launch
  const bool mine = G.single ? m < P.M : live_flag;
  const bool live = live_flag;
  const long long off = P.off0 + (long long)m * P.n + tk.row0;
  double rv[R], zp[R];
  double bn = 0.0, rrv = 0.0, tolm = 0.0, xxv = 0.0, jxv = 0.0;
  int itj = 0;
  TS cw[kCwPerLane];  // c_c w_c for c = lane + 32 j
#pragma unroll
  for (int j = 0; j < kCwPerLane; ++j) cw[j] = TS(0);
  if (mine) {
    if (!init) {
      bn = sc[item].bnorm;
      rrv = acc[item].rr;
      itj = sc[item].iters + 1;
      tolm = sc[item].tolm;
      if (P.etol > 0.0) xxv = acc[item].xx;
      if (P.jhist != nullptr) jxv = acc[item].jx;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = lane + 32 * j;
      if (i < tk.rows) {
        rv[j] = r[off + i];
        if (zpre != nullptr) zp[j] = zpre[off + i];
      }
    }
#pragma unroll
    for (int j = 0; j < kCwPerLane; ++j) {
      const int c = lane + 32 * j;
      if (c < k) cw[j] = (TS)(P.c[c] * (double)Wk[(long long)item * kmax + c]);
    }
  }
  const TS* S = static_cast<const TS*>(P.S);
  stage_S<TS>(S, P.n, k, tk.row0, tk.rows, Ssm, 1, KP);
  if (k > 0)
    for (int idx = threadIdx.x; idx < tk.rows * (KP - k); idx += kThreads) {
      const int i = idx / (KP - k);
      Ssm[i * KP + k + (idx - i * (KP - k))] = TS(0);
    }
  // p^T q of the next sweep accumulates from zero
  if (tk.first && blockIdx.y == 0)
    for (int mm = threadIdx.x; mm < P.M; mm += kThreads) acc[P.item0 + mm].pq = 0.0;
  __syncthreads();
  if (!live) return;
  const int slot = init ? 0 : (par ^ 1);
  TS* wc = wsm + wid * KW;
  if (!init) {
    // the stopping test, from values no CTA of this launch writes
    const double rel = bn > 0.0 ? sqrt(rrv) / bn : 0.0;
    bool stop = false;
    int st = EDA_MAXIT;
    if (!isfinite(rel)) {
      st = EDA_NAN;
      stop = true;
    } else if (fixed > 0) {
      if (itj >= fixed) {
        st = EDA_CONVERGED;
        stop = true;
      }
    } else {
      // every requested criterion: the relative residual (tol > 0) and the
      // certified error bound ||r|| / (||x|| - ||r||) (etol > 0); or the
      // inner threshold tolm of a refinement round
      bool fin = !(tol > 0.0) || rel <= tol;
      if (P.etol > 0.0) {
        const double rn = rel * bn, xn = sqrt(xxv);
        fin = fin && xn > rn && rn <= P.etol * (xn - rn);
      }
      if (fin || (tolm > 0.0 && rel <= tolm)) {
        st = EDA_CONVERGED;
        stop = true;
      } else if (maxit > 0 && itj >= maxit) {
        stop = true;
      }
    }
    if (tk.first && lane == 0) {
      sc[item].relres = rel;
      if (P.jhist != nullptr) {
        // this launch's only reader of jx: record, then clear for the next update
        if (itj < P.jstride) P.jhist[(long long)m * P.jstride + itj] = -0.5 * jxv;
        acc[item].jx = 0.0;
      }
      acc[item].inc = 1;
      if (stop) {
        sc[item].status = st;
        active[item] = 0;
        atomicSub(nactive, 1);
      }
    }
    if (stop) return;
  }
#pragma unroll
  for (int j = 0; j < kCwPerLane; ++j)
    if (lane + 32 * j < KP) wc[lane + 32 * j] = cw[j];
  __syncwarp();
  double rz = 0.0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int i = lane + 32 * j;
    if (i < tk.rows) {
      double zv = zpre != nullptr ? zp[j] : rv[j];
      if (k > 0) {
        const V* Srow = reinterpret_cast<const V*>(Ssm + i * KP);
        const V* wv = reinterpret_cast<const V*>(wc);
        TS s0 = 0, s1 = 0;
        int c = 0;
        for (; c + 2 <= KP / VW; c += 2) {
          s0 += Vec16<TS>::dot(Srow[c], wv[c]);
          s1 += Vec16<TS>::dot(Srow[c + 1], wv[c + 1]);
        }
        if (c < KP / VW) s0 += Vec16<TS>::dot(Srow[c], wv[c]);
        zv += (double)(s0 + s1);
      }
      z[off + i] = zv;
      if (init) p[off + i] = zv;
      rz += rv[j] * zv;
    }
  }
  rz = warp_sum(rz);
  if (lane == 0) atomicAdd(&acc[item].rz[slot], rz);
}

template <typename TS>
__global__ void __launch_bounds__(kThreads) pcg2_dir_kernel(const PcgGrid G, int kmax,
                                                            const double* z, double* p, PcgScalars* sc, PcgAcc* acc,
                                                            const int* active, TS* Wk, int par,
                                                            const int* nactive, int* host_count) {
  PcgTask tk;
  PcgProb P;
  grid_task(G, &tk, &P);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // the active count is final here (update and precond change it): one
  // thread copies it to the host's ring slot (mapped pinned memory)
  if (host_count != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    *reinterpret_cast<volatile int*>(host_count) = *nactive;
  if (tk.first && blockIdx.y == 0) {
    // bookkeeping of the problem: iteration counts, and the accumulators
    // the next update launch fills
    for (int m = threadIdx.x; m < P.M; m += kThreads) {
      const int item = P.item0 + m;
      if (acc[item].inc) {
        sc[item].iters += 1;
        acc[item].inc = 0;
      }
      acc[item].rr = 0.0;
      acc[item].xx = 0.0;
    }
    for (int idx = threadIdx.x; idx < P.M * kmax; idx += kThreads)
      Wk[(long long)P.item0 * kmax + idx] = TS(0);
  }
  {
    const int m = blockIdx.y * kWarps + wid;  // one member per warp
    if (m >= P.M) return;
    const int item = P.item0 + m;
    // a handle's solve has every load in flight before the active flag is
    // tested (see the update launch); the group path tests it first
    if (!G.single && !active[item]) return;
    constexpr int R = kRowsPerLane;
    const long long off = P.off0 + (long long)m * P.n + tk.row0;
    double zv[R], pv[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = lane + 32 * j;
      if (i < tk.rows) {
        zv[j] = z[off + i];
        pv[j] = p[off + i];
      }
    }
    const double rzn = acc[item].rz[par ^ 1], rzo = acc[item].rz[par];
    if (!active[item]) return;
    const double beta = rzn / rzo;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = lane + 32 * j;
      if (i < tk.rows) p[off + i] = zv[j] + beta * pv[j];
    }
  }
}

// r = b - hx and ||r||^2 for the active members (hx = (I + A) x).
__global__ void __launch_bounds__(kThreads) pcg2_replace_kernel(const PcgGrid G, const double* b, const double* hx, double* r,
                                                                PcgAcc* acc, const int* active) {
  PcgTask tk;
  PcgProb P;
  grid_task(G, &tk, &P);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int m = blockIdx.y * kWarps + wid;
  if (m >= P.M) return;
  const int item = P.item0 + m;
  if (!active[item]) return;
  const long long off = P.off0 + (long long)m * P.n + tk.row0;
  double rr = 0.0;
  for (int i = lane; i < tk.rows; i += 32) {
    const double rv = b[off + i] - hx[off + i];
    r[off + i] = rv;
    rr += rv * rv;
  }
  rr = warp_sum(rr);
  if (lane == 0) atomicAdd(&acc[item].rr, rr);
}

__global__ void pcg2_reset_kernel(PcgAcc* acc, int T) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x) {
    PcgAcc a;
    a.pq = a.rr = a.rz[0] = a.rz[1] = a.xx = a.jx = 0.0;
    a.inc = a.pad = 0;
    acc[j] = a;
  }
}

__global__ void pcg2_col_dot_kernel(int n, const double* v, const double* hv, const int* active, PcgAcc* acc) {
  __shared__ double red[kWarps];
  const int col = blockIdx.y;
  if (active && !active[col]) return;
  const long long base = (long long)col * n;
  double s = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) s += v[base + i] * hv[base + i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    atomicAdd(&acc[col].pq, t);
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

PcgGrid pcg_single(const PcgProb& prob) {
  PcgGrid g{};
  g.single = 1;
  g.one = prob;
  g.ntasks = (prob.n + kPcgRows - 1) / kPcgRows;
  return g;
}

PcgGrid pcg_tables(const PcgTask* tasks, int ntasks, const PcgProb* probs) {
  PcgGrid g{};
  g.tasks = tasks;
  g.probs = probs;
  g.ntasks = ntasks;
  return g;
}

void pcg_tasks(const int* n_of, int nprob, std::vector<PcgTask>* out) {
  out->clear();
  for (int pi = 0; pi < nprob; ++pi)
    for (int r0 = 0; r0 < n_of[pi]; r0 += kPcgRows) {
      const int rows = (n_of[pi] - r0 < kPcgRows) ? n_of[pi] - r0 : kPcgRows;
      out->push_back(PcgTask{pi, r0, rows, r0 == 0 ? 1 : 0});
    }
}

cudaError_t pcg2_reset(PcgAcc* acc, int T, void* Wk, size_t wk_bytes, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  count_launch();
  pcg2_reset_kernel<<<(T + 255) / 256, 256, 0, s>>>(acc, T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || wk_bytes == 0) return e;
  return cudaMemsetAsync(Wk, 0, wk_bytes, s);
}

template <typename TS>
cudaError_t pcg2_update(const PcgGrid& G, int kmax, int mmax, const double* p,
                        const double* q, double* x, double* r, PcgScalars* sc, PcgAcc* acc, int* active, TS* Wk,
                        int par, int update, int use_lmp, int* nactive, cudaStream_t s) {
  if (G.ntasks <= 0 || mmax <= 0) return cudaSuccess;
  const size_t smem = ((size_t)kmax * vec_stride<TS>(kPcgRows) + (size_t)kWarps * kPcgRows) * sizeof(TS);
  cudaError_t e = set_smem(pcg2_update_kernel<TS>, smem);
  if (e != cudaSuccess) return e;
  count_launch();
  pcg2_update_kernel<TS><<<dim3(G.ntasks, (mmax + kWarps - 1) / kWarps), kThreads, smem, s>>>(G, kmax, p, q, x, r, sc, acc, active, Wk, par,
                                                        update, use_lmp, nactive);
  return cudaGetLastError();
}

template <typename TS>
cudaError_t pcg2_precond(const PcgGrid& G, int kmax, int mmax, const double* r,
                         double* z, double* p, PcgScalars* sc, PcgAcc* acc, int* active, const TS* Wk, int par,
                         double tol, int maxit, int fixed, int use_lmp, int init, int* nactive, cudaStream_t s,
                         const double* zpre) {
  if (G.ntasks <= 0 || mmax <= 0) return cudaSuccess;
  if (vec_stride<TS>(kmax) > 32 * kCwPerLane) return cudaErrorInvalidValue;  // more than 80 LMP modes
  const int KW = vec_stride<TS>(kmax > 0 ? kmax : 1);
  const size_t smem = ((size_t)kPcgRows * KW + (size_t)kWarps * KW) * sizeof(TS);
  cudaError_t e = set_smem(pcg2_precond_kernel<TS>, smem);
  if (e != cudaSuccess) return e;
  count_launch();
  pcg2_precond_kernel<TS><<<dim3(G.ntasks, (mmax + kWarps - 1) / kWarps), kThreads, smem, s>>>(G, kmax, r, z, p, sc, acc, active, Wk, par, tol,
                                                         maxit, fixed, use_lmp, init, nactive, zpre);
  return cudaGetLastError();
}

template <typename TS>
cudaError_t pcg2_dir(const PcgGrid& G, int kmax, int mmax, const double* z, double* p,
                     PcgScalars* sc, PcgAcc* acc, const int* active, TS* Wk, int par, cudaStream_t s,
                     const int* nactive, int* host_count) {
  if (G.ntasks <= 0 || mmax <= 0) return cudaSuccess;
  count_launch();
  pcg2_dir_kernel<TS><<<dim3(G.ntasks, (mmax + kWarps - 1) / kWarps), kThreads, 0, s>>>(G, kmax, z, p, sc, acc,
                                                                                     active, Wk, par, nactive,
                                                                                     host_count);
  return cudaGetLastError();
}

cudaError_t pcg2_replace(const PcgGrid& G, int mmax, const double* b,
                         const double* hx, double* r, PcgAcc* acc, int T, const int* active, cudaStream_t s) {
  if (G.ntasks <= 0 || mmax <= 0) return cudaSuccess;
  // ||r||^2 of the replaced residual accumulates from zero
  cudaError_t e = cudaMemset2DAsync(&acc[0].rr, sizeof(PcgAcc), 0, sizeof(double), T, s);
  if (e != cudaSuccess) return e;
  count_launch();
  pcg2_replace_kernel<<<dim3(G.ntasks, (mmax + kWarps - 1) / kWarps), kThreads, 0, s>>>(G, b, hx, r, acc,
                                                                                      active);
  return cudaGetLastError();
}

cudaError_t pcg2_col_dot(int n, int ncol, const double* v, const double* hv, const int* active, PcgAcc* acc,
                         cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  int bx = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (bx > 64) bx = 64;
  count_launch();
  pcg2_col_dot_kernel<<<dim3(bx, ncol), kThreads, 0, s>>>(n, v, hv, active, acc);
  return cudaGetLastError();
}

template cudaError_t pcg2_update<double>(const PcgGrid&, int, int, const double*, const double*,
                                         double*, double*, PcgScalars*, PcgAcc*, int*, double*, int, int, int, int*,
                                         cudaStream_t);
template cudaError_t pcg2_update<float>(const PcgGrid&, int, int, const double*, const double*,
                                        double*, double*, PcgScalars*, PcgAcc*, int*, float*, int, int, int, int*,
                                        cudaStream_t);
template cudaError_t pcg2_precond<double>(const PcgGrid&, int, int, const double*, double*, double*,
                                          PcgScalars*, PcgAcc*, int*, const double*, int, double, int, int, int,
                                          int, int*, cudaStream_t, const double*);
template cudaError_t pcg2_precond<float>(const PcgGrid&, int, int, const double*, double*, double*,
                                         PcgScalars*, PcgAcc*, int*, const float*, int, double, int, int, int, int,
                                         int*, cudaStream_t, const double*);
template cudaError_t pcg2_dir<double>(const PcgGrid&, int, int, const double*, double*, PcgScalars*,
                                      PcgAcc*, const int*, double*, int, cudaStream_t, const int*, int*);
template cudaError_t pcg2_dir<float>(const PcgGrid&, int, int, const double*, double*, PcgScalars*,
                                     PcgAcc*, const int*, float*, int, cudaStream_t, const int*, int*);

}  // namespace eda
