// Lorenz-96 sweeps on sm_103a: nonlinear trajectory with innovations, the
// tangent-linear/adjoint Hessian-vector product (I + A) v, and the adjoint
// right-hand side U_B^T G^T R^{-1} d (Section 2.3, Eq. (system with CVT);
// the model and RK4 step of Section 4).
//
// Layout of one column (one vector on one member's trajectory), sweep_kernel:
//  * the column is split over a thread-block cluster of CS CTAs; CTA r owns
//    the global indices [r*Ttile, min((r+1)*Ttile, n));
//  * each CTA computes on an extended region of E = A*C consecutive (periodic)
//    indices starting HL before its tile; thread t keeps elements
//    [t*C, t*C + C) of that region in registers;
//  * a stage of RK4 needs the neighbours i-2, i-1, i+1, i+2 of a thread's
//    run: threads publish the first two and last two values of their run to
//    a shared-memory edge buffer and read their neighbours' after a barrier;
//  * the stencil wraps inside the extended region, so values near its ends
//    go wrong (an error from outside travels at most 8 points per
//    tangent-linear step and 11 per adjoint step, 8K + 3 over K steps);
//    every K steps the halo is reloaded from its owners (distributed shared
//    memory inside the cluster), and HL = 8K + 8 keeps the owned tile exact
//    (for CS = 1 the owner is the CTA itself and the reload implements the
//    periodic boundary);
//  * trajectory runs are loaded straight into registers with 16-byte loads,
//    one step ahead; the FP64 variant (STG) reads the RK4 stage states
//    stored with the trajectory instead of recomputing them;
//  * the Hessian-product epilogue applies U_B from the cluster's mirrors and
//    adds v . (H v) of the column to the PCG accumulators.
// Columns too long for one cluster run as chains of K-step launches whose
// state passes through global buffers (multi-launch tiling, launch_sweep).
// wsweep_kernel, the warp-tiled Hessian-product variant, is described where
// it is defined.
//
// The tangent linear is the exact derivative of the discrete RK4 step and
// the adjoint its exact transpose, computed stage by stage in reverse.
#include <cooperative_groups.h>

#include <cstdio>
#include <cstdlib>

#include "eda_internal.h"
#include "pcg.h"

namespace cg = cooperative_groups;

namespace eda {
namespace {

constexpr int kNumEdge = 6;
constexpr int kMaxThreads = 512;

template <typename T, int C>
struct Run {
  T v[C];
  T m2, m1, p1, p2;
  // Element j of the run, j in [-2, C+1]; j is a compile-time constant after
  // unrolling so this folds to a register.
  __device__ __forceinline__ T at(int j) const {
    return j == -2 ? m2
                   : (j == -1 ? m1
                              : (j == C ? p1 : (j == C + 1 ? p2 : v[j < 0 ? 0 : (j >= C ? C - 1 : j)])));
  }
};

// Lorenz-96 tendency f_j = (x_{j+1} - x_{j-2}) x_{j-1} - x_j + F.
template <typename T, int C>
__device__ __forceinline__ T tend(const Run<T, C>& X, int j, T F) {
  return (X.at(j + 1) - X.at(j - 2)) * X.at(j - 1) - X.at(j) + F;
}
// (J(X) e)_j = (e_{j+1} - e_{j-2}) X_{j-1} + (X_{j+1} - X_{j-2}) e_{j-1} - e_j.
template <typename T, int C>
__device__ __forceinline__ T jvp(const Run<T, C>& X, const Run<T, C>& e, int j) {
  return (e.at(j + 1) - e.at(j - 2)) * X.at(j - 1) + (X.at(j + 1) - X.at(j - 2)) * e.at(j - 1) - e.at(j);
}
// (J(X)^T w)_j = X_{j-2} w_{j-1} + (X_{j+2} - X_{j-1}) w_{j+1} - X_{j+1} w_{j+2} - w_j.
template <typename T, int C>
__device__ __forceinline__ T jtvp(const Run<T, C>& X, const Run<T, C>& w, int j) {
  return X.at(j - 2) * w.at(j - 1) + (X.at(j + 2) - X.at(j - 1)) * w.at(j + 1) - X.at(j + 1) * w.at(j + 2) -
         w.at(j);
}

// The stencils with the stored difference D_j = X_{j+1} - X_{j-2} of the
// state (three FP64 instructions each instead of five):
// (J(X) e)_j = (e_{j+1} - e_{j-2}) X_{j-1} + D_j e_{j-1} - e_j, with
// xm1 = X_{j-1} and d = D_j;
template <typename T, int C>
__device__ __forceinline__ T jvpd(T xm1, T d, const Run<T, C>& e, int j) {
  return fma(e.at(j + 1) - e.at(j - 2), xm1, fma(d, e.at(j - 1), -e.at(j)));
}
// (J(X)^T w)_j = X_{j-2} w_{j-1} + D_{j+1} w_{j+1} - X_{j+1} w_{j+2} - w_j,
// with dp1 = D_{j+1}.
template <typename T, int C>
__device__ __forceinline__ T jtvpd(const Run<T, C>& X, T dp1, const Run<T, C>& w, int j) {
  return fma(X.at(j - 2), w.at(j - 1), fma(dp1, w.at(j + 1), fma(-X.at(j + 1), w.at(j + 2), -w.at(j))));
}

// Reverse RK4 step.  The TL step is e' = e + h/6 (k1 + 2 k2 + 2 k3 + k4),
// k_s = J_s e_s, e_1 = e, e_2 = e + h/2 k1, e_3 = e + h/2 k2, e_4 = e + h k3.
// Its adjoint maps lam (the weight of e') to
//   lam + h/6 u4 + h/3 u3 + h/3 u2 + h/6 u1,   u_s = J_s^T b_s,
//   b4 = lam, b3 = lam + h/2 u4, b2 = lam + h/2 u3, b1 = lam + h u2,
// which is the textbook recursion (stage weights a4 = h/6 lam,
// a3 = h/3 lam + h J4^T a4, a2 = h/3 lam + h/2 J3^T a3,
// a1 = h/6 lam + h/2 J2^T a2) with a_s = h/6 b4, h/3 b3, h/3 b2, h/6 b1
// factored out by linearity: one FMA per weight and per accumulated slope.

struct Geo {
  // A: threads holding the extended region (the neighbour wrap); AS: edge
  // buffer slot stride and NT: loop stride (both the block size)
  int n, E, A, AS, NT, tid, tl, tr, l0, HL, Ttile, Town, a0, gbase, CS, rank;
};

template <typename T, int C>
__device__ __forceinline__ void publish(T* eb, const Geo& g, const T (&v)[C]) {
  eb[g.tid] = v[0];
  eb[g.AS + g.tid] = v[1];
  eb[2 * g.AS + g.tid] = v[C - 2];
  eb[3 * g.AS + g.tid] = v[C - 1];
}

template <typename T, int C>
__device__ __forceinline__ void fetch(const T* eb, const Geo& g, Run<T, C>& r) {
  r.m2 = eb[2 * g.AS + g.tl];
  r.m1 = eb[3 * g.AS + g.tl];
  r.p1 = eb[g.tr];
  r.p2 = eb[g.AS + g.tr];
}

// Run of the stage buffer xs (whole extended region resident in smem).
template <typename T, int C>
__device__ __forceinline__ void run_from_smem(const T* xs, const Geo& g, Run<T, C>& r) {
#pragma unroll
  for (int c = 0; c < C; ++c) r.v[c] = xs[g.l0 + c];
  r.m2 = xs[g.l0 >= 2 ? g.l0 - 2 : g.l0 - 2 + g.E];
  r.m1 = xs[g.l0 >= 1 ? g.l0 - 1 : g.l0 - 1 + g.E];
  r.p1 = xs[g.l0 + C < g.E ? g.l0 + C : g.l0 + C - g.E];
  r.p2 = xs[g.l0 + C + 1 < g.E ? g.l0 + C + 1 : g.l0 + C + 1 - g.E];
}

__device__ __forceinline__ void sync_cluster_or_block(bool cluster) {
  if (cluster) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// Reads the halo elements of v (positions outside the owned tile) from their
// owners' mirrors.  The caller has written every thread's v to its own
// mirror and passed a cluster (or block) barrier.
template <typename T, int C>
__device__ __forceinline__ void read_halo(T (&v)[C], T* mir, const Geo& g) {
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int l = g.l0 + c;
    if (l < g.HL || l >= g.HL + g.Town) {
      const int gi = (g.gbase + l) % g.n;
      const int r2 = gi / g.Ttile;
      const int ll = g.HL + gi - r2 * g.Ttile;
      if (g.CS == 1 || r2 == g.rank) {
        v[c] = mir[ll];
      } else {
        const T* rem = cg::this_cluster().map_shared_rank(mir, r2);
        v[c] = rem[ll];
      }
    }
  }
}

// Observation k-ranges of a CTA at observation step oj (see obs_table), from
// the CTA's rows of the table (tabp: shared memory, or global when they do
// not fit).
__device__ __forceinline__ const int* obs_ranges(const int* tabp, int oj) { return tabp + oj * 8; }

// Own run <-> mirror, with 16-byte shared-memory accesses (8-byte ones for a
// run of two FP32 values).
template <typename T, int C>
__device__ __forceinline__ void write_mirror(T* mir, const Geo& g, const T (&v)[C]) {
  static_assert((C * sizeof(T)) % 8 == 0, "run must be a whole number of 8-byte chunks");
  if constexpr (sizeof(T) == 4 && C % 4 != 0) {
    float2* p = reinterpret_cast<float2*>(mir + g.l0);
#pragma unroll
    for (int q = 0; q < C / 2; ++q) p[q] = make_float2(v[2 * q], v[2 * q + 1]);
  } else if constexpr (sizeof(T) == 4) {
    float4* p = reinterpret_cast<float4*>(mir + g.l0);
#pragma unroll
    for (int q = 0; q < C / 4; ++q) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
    double2* p = reinterpret_cast<double2*>(mir + g.l0);
#pragma unroll
    for (int q = 0; q < C / 2; ++q) p[q] = make_double2(v[2 * q], v[2 * q + 1]);
  }
}

template <typename T, int C>
__device__ __forceinline__ void write_mirror_zero(T* mir, const Geo& g) {
  T z[C];
#pragma unroll
  for (int c = 0; c < C; ++c) z[c] = T(0);
  write_mirror<T, C>(mir, g, z);
}

template <typename T, int C>
__device__ __forceinline__ void add_mirror(const T* mir, const Geo& g, T (&v)[C]) {
  if constexpr (sizeof(T) == 4 && C % 4 != 0) {
    const float2* p = reinterpret_cast<const float2*>(mir + g.l0);
#pragma unroll
    for (int q = 0; q < C / 2; ++q) {
      const float2 u = p[q];
      v[2 * q] += u.x;
      v[2 * q + 1] += u.y;
    }
  } else if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(mir + g.l0);
#pragma unroll
    for (int q = 0; q < C / 4; ++q) {
      const float4 u = p[q];
      v[4 * q] += u.x;
      v[4 * q + 1] += u.y;
      v[4 * q + 2] += u.z;
      v[4 * q + 3] += u.w;
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(mir + g.l0);
#pragma unroll
    for (int q = 0; q < C / 2; ++q) {
      const double2 u = p[q];
      v[2 * q] += u.x;
      v[2 * q + 1] += u.y;
    }
  }
}

// mir[obs_idx[k] - base] = stash[k] for k in [k0, k1), four loads in flight
// per thread.
template <typename T>
__device__ __forceinline__ void scatter_obs(const int* __restrict__ idx, const T* __restrict__ stash, int k0,
                                            int k1, int base, int tid, int A, T* mir) {
  for (int k = k0 + tid; k < k1; k += 4 * A) {
    int ii[4];
    T vv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int kk = k + u * A;
      ii[u] = kk < k1 ? __ldg(idx + kk) : 0;
      vv[u] = kk < k1 ? __ldcg(stash + kk) : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k + u * A < k1) mir[ii[u] - base] = vv[u];
  }
}

// out[c] = sum_{|d|<=w} cf[|d|] src[base + w + c + d] for c < C: the banded
// symmetric circulant on C consecutive outputs with a sliding register window
// (3 shared-memory loads per tap).  src holds the input with a w-halo.
template <typename T, int C>
__device__ __forceinline__ void conv_run(const T* src, int base, int w, const T* cf, T (&out)[C]) {
  T Lw[C], Rw[C];
  const T c0 = cf[0];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    Lw[c] = src[base + w + c];
    Rw[c] = Lw[c];
    out[c] = c0 * Lw[c];
  }
  for (int d = 1; d <= w; ++d) {
#pragma unroll
    for (int c = C - 1; c > 0; --c) Lw[c] = Lw[c - 1];
    Lw[0] = src[base + w - d];
#pragma unroll
    for (int c = 0; c < C - 1; ++c) Rw[c] = Rw[c + 1];
    Rw[C - 1] = src[base + w + C - 1 + d];
    const T cd = cf[d];
#pragma unroll
    for (int c = 0; c < C; ++c) out[c] += cd * (Lw[c] + Rw[c]);
  }
}

// U_B lambda on the owned tile from the mirrors of the cluster (+ v if ident);
// thread t produces outputs [t*C, t*C + C) of the tile.  stage has room for
// E + 2w values.
template <typename T, int C, typename TO>
__device__ void bhalf_from_mirrors(const SweepArgs<T>& a, const Geo& g, T* mir, T* stage, const T* cf,
                                   TO* out, const double* ident64, const T* ident, double* dot) {
  const int w = a.w;
  const int cnt = g.Town + 2 * w;
  for (int j = g.tid; j < cnt; j += g.NT) {
    int gi = (g.a0 - w + j) % g.n;
    if (gi < 0) gi += g.n;
    const int r2 = gi / g.Ttile;
    const int ll = g.HL + gi - r2 * g.Ttile;
    if (g.CS == 1 || r2 == g.rank) {
      stage[j] = mir[ll];
    } else {
      const T* rem = cg::this_cluster().map_shared_rank(mir, r2);
      stage[j] = rem[ll];
    }
  }
  // every remote read of this cluster's mirrors is complete after this barrier
  sync_cluster_or_block(g.CS > 1);
  const int j0 = g.tid * C;
  double part = 0.0;  // v . (H v) over this thread's outputs
  if (j0 < g.Town) {
    T o[C];
    conv_run<T, C>(stage, j0, w, cf, o);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (j0 + c < g.Town) {
        TO v = (TO)o[c];
        double in = 0.0;
        if (ident64) in = ident64[g.a0 + j0 + c];
        else if (ident) in = (double)ident[g.a0 + j0 + c];
        if (ident64 || ident) v += (TO)in;
        out[g.a0 + j0 + c] = v;
        part += in * (double)v;
      }
    }
  }
  if (dot != nullptr) {  // uniform over the CTA
    // the mirror is free here: every remote read of it ended at the cluster
    // barrier above, and the outputs were taken from the stage area
    double* red = reinterpret_cast<double*>(mir);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((g.tid & 31) == 0) red[g.tid >> 5] = part;
    __syncthreads();
    if (g.tid == 0) {
      double t = 0.0;
      for (int i = 0; i < g.NT / 32; ++i) t += red[i];
      atomicAdd(dot, t);
    }
  }
}

// stash[k] = R^{-1}_k delta_t[obs_idx[k]] for the observations of the owned
// tile at observation step oj; the owned values are in the mirror.
template <typename T>
__device__ __forceinline__ void gather_obs(const SweepArgs<T>& a, const Geo& g, int oj, const int* tabp, const T* mir,
                                           T* stash) {
  if (tabp != nullptr) {
    const int* tb = obs_ranges(tabp, oj);
    const int k0 = tb[0], k1 = tb[1];
    const int off = g.HL - g.a0;
    for (int k = k0 + g.tid; k < k1; k += 4 * g.NT) {
      int ii[4];
      T rr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = k + u * g.NT;
        ii[u] = kk < k1 ? __ldg(a.obs_idx + kk) : 0;
        rr[u] = kk < k1 ? __ldg(a.rinv + kk) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u * g.NT < k1) stash[k + u * g.NT] = rr[u] * mir[off + ii[u]];
    }
  } else {
    const int k0 = a.obs_ptr[oj], k1 = a.obs_ptr[oj + 1];
    for (int k = k0 + g.tid; k < k1; k += g.NT) {
      const int gi = a.obs_idx[k];
      if (gi >= g.a0 && gi < g.a0 + g.Town) stash[k] = a.rinv[k] * mir[g.HL + gi - g.a0];
    }
  }
}

// Observation loads of one gather or injection issued a step ahead: the
// first kObsPre observations of each thread's share (k = first + tid + u NT)
// go to registers at the start of the step that ends with the gather or
// injection, which then takes the rest with direct loads.
constexpr int kObsPre = 2;

template <typename T>
struct ObsPre {
  int idx[kObsPre];
  T val[kObsPre];
};

// Gather of the owned tile at observation step oj: obs_idx and R^{-1}.
template <typename T>
__device__ __forceinline__ void gather_pre(const SweepArgs<T>& a, const Geo& g, const int* tb, ObsPre<T>& q) {
#pragma unroll
  for (int u = 0; u < kObsPre; ++u) {
    const int k = tb[0] + g.tid + u * g.NT;
    q.idx[u] = k < tb[1] ? __ldg(a.obs_idx + k) : 0;
    q.val[u] = k < tb[1] ? __ldg(a.rinv + k) : T(0);
  }
}

// stash[k] = R^{-1}_k delta[obs_idx[k]] (as gather_obs) from the prefetched
// loads and direct loads for the rest.
template <typename T>
__device__ __forceinline__ void gather_use(const SweepArgs<T>& a, const Geo& g, const int* tb, const ObsPre<T>& q,
                                           const T* mir, T* stash) {
  const int off = g.HL - g.a0;
#pragma unroll
  for (int u = 0; u < kObsPre; ++u) {
    const int k = tb[0] + g.tid + u * g.NT;
    if (k < tb[1]) stash[k] = q.val[u] * mir[off + q.idx[u]];
  }
  for (int k = tb[0] + g.tid + kObsPre * g.NT; k < tb[1]; k += g.NT)
    stash[k] = __ldg(a.rinv + k) * mir[off + __ldg(a.obs_idx + k)];
}

// Injection over the extended region at observation step oj: its two index
// segments (k0, k1, base) as one sequence j = 0 .. cnt-1.
__device__ __forceinline__ void inject_k(const int* tb, int j, int* k, int* base) {
  const int ca = tb[3] - tb[2];
  *k = j < ca ? tb[2] + j : tb[5] + (j - ca);
  *base = j < ca ? tb[4] : tb[7];
}

template <typename T>
__device__ __forceinline__ void inject_pre(const SweepArgs<T>& a, const Geo& g, const int* tb, const T* stash,
                                           ObsPre<T>& q) {
  const int cnt = (tb[3] - tb[2]) + (tb[6] - tb[5]);
#pragma unroll
  for (int u = 0; u < kObsPre; ++u) {
    const int j = g.tid + u * g.NT;
    int k, base;
    inject_k(tb, j, &k, &base);
    q.idx[u] = j < cnt ? __ldg(a.obs_idx + k) : 0;
    q.val[u] = j < cnt ? __ldcg(stash + k) : T(0);
  }
}

// mir[obs_idx[k] - base] = stash[k] (as scatter_obs over both segments).
template <typename T>
__device__ __forceinline__ void inject_use(const SweepArgs<T>& a, const Geo& g, const int* tb, const ObsPre<T>& q,
                                           const T* stash, T* mir) {
  const int cnt = (tb[3] - tb[2]) + (tb[6] - tb[5]);
#pragma unroll
  for (int u = 0; u < kObsPre; ++u) {
    const int j = g.tid + u * g.NT;
    int k, base;
    inject_k(tb, j, &k, &base);
    if (j < cnt) mir[q.idx[u] - base] = q.val[u];
  }
  for (int j = g.tid + kObsPre * g.NT; j < cnt; j += g.NT) {
    int k, base;
    inject_k(tb, j, &k, &base);
    mir[__ldg(a.obs_idx + k) - base] = __ldcg(stash + k);
  }
}

// Own run of the trajectory state at row `row` (C consecutive elements of the
// extended region): one or two 16-byte vector loads when aligned, else scalar.
template <typename T, int C>
__device__ __forceinline__ void load_run(const T* row, const int (&gi)[C], bool vec_ok, T (&out)[C]) {
  if (vec_ok) {
    if constexpr (sizeof(T) == 4 && C % 4 != 0) {
      const float2* p = reinterpret_cast<const float2*>(row + gi[0]);
#pragma unroll
      for (int v = 0; v < C / 2; ++v) {
        const float2 q = __ldg(p + v);
        out[2 * v] = q.x;
        out[2 * v + 1] = q.y;
      }
    } else if constexpr (sizeof(T) == 4) {
      const float4* p = reinterpret_cast<const float4*>(row + gi[0]);
#pragma unroll
      for (int v = 0; v < C / 4; ++v) {
        const float4 q = __ldg(p + v);
        out[4 * v] = q.x;
        out[4 * v + 1] = q.y;
        out[4 * v + 2] = q.z;
        out[4 * v + 3] = q.w;
      }
    } else {
      const double2* p = reinterpret_cast<const double2*>(row + gi[0]);
#pragma unroll
      for (int v = 0; v < C / 2; ++v) {
        const double2 q = __ldg(p + v);
        out[2 * v] = q.x;
        out[2 * v + 1] = q.y;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) out[c] = __ldg(row + gi[c]);
  }
}

// A column whose trajectory index lies outside the store [0, M) (M > 0):
// the caller passed a bad member_of_col.  Its outputs become NaN and no
// trajectory row is read.
template <typename T>
__device__ __forceinline__ bool bad_member(const SweepArgs<T>& a, int member) {
  return a.M > 0 && (unsigned)member >= (unsigned)a.M;
}

// NaN over the owned tile of a column's output: the state buffer of a
// multi-launch chain (its closing U_B kernel then writes NaN), else the
// output vector.
template <typename T>
__device__ void nan_owned(const SweepArgs<T>& a, const Geo& g, int col, long long voff) {
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if (a.ml) {
    if (a.st_out != nullptr)
      for (int j = g.tid; j < g.Town; j += g.NT) a.st_out[(long long)col * a.n + g.a0 + j] = (T)qnan;
    return;
  }
  for (int j = g.tid; j < g.Town; j += g.NT) {
    if (a.OUT64 != nullptr) a.OUT64[voff + g.a0 + j] = qnan;
    else if (a.OUT != nullptr) a.OUT[voff + g.a0 + j] = (T)qnan;
  }
}

constexpr int kObsMapCap = 1024;  // steps whose observation index is cached in smem
constexpr int kObsTabCap = 2048;  // entries of a CTA's observation range rows cached in smem

// STG: the kernel reads stored stage states when the arguments carry them
// (instantiated for FP64 only: FP32 sweeps recompute, which costs them less
// than streaming three more arrays).
// CK: the kernel recomputes its launch's states from a checkpointed
// trajectory (multi-launch plans with ckpt > 0; never with STG).
// One column's sweep by this CTA (the body of sweep_kernel and of the
// persistent PCG kernel, which calls it once per iteration).
template <typename T, int C, bool STG, bool CK>
__device__ __forceinline__ void sweep_body(const SweepArgs<T>& a0, const int col) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);

  SweepArgs<T> a = a0;
  Geo g;
  g.CS = a.CS;
  g.rank = (a.CS > 1) ? (a.ml ? (int)(blockIdx.x % a.CS) : (int)cg::this_cluster().block_rank()) : 0;
  if (col >= a.ncol) return;
  // launch-wide shared-memory layout (the group launch sizes it for its largest problem)
  const int Emax = (int)blockDim.x * C;
  const int wmax = a0.w;
  int member, A_act = (int)blockDim.x;
  int item = col;  // accumulator index of the column (dot_out)
  long long voff, soff;
  if (a.items != nullptr) {
    const SweepItem it = a.items[col];
    item = it.flag;
    if (it.flag >= 0 && a.flags[it.flag] == 0) return;  // uniform over the cluster
    const SweepProb<T> P = a.probs[it.prob];
    a.n = P.n;
    a.N = P.N;
    a.p = P.p;
    a.w = P.w;
    a.nos = P.nos;
    a.Ttile = P.Ttile;
    a.HL = P.HL;
    a.E = P.E;
    a.K = P.K;
    a.F = P.F;
    a.dt = P.dt;
    a.traj = P.traj;
    a.traj_mstride = P.traj_mstride;
    a.obs_of_t = P.obs_of_t;
    a.obs_ptr = P.obs_ptr;
    a.obs_idx = P.obs_idx;
    a.rinv = P.rinv;
    a.obs_tab = P.obs_tab;
    a.bcoef = P.bcoef;
    member = it.member;
    voff = it.voff;
    soff = it.soff;
    A_act = P.A;
    if (a.mode == MODE_NL && a.traj_out != nullptr) {
      a.traj_out = const_cast<T*>(P.traj);
      a.traj_out_mstride = P.traj_mstride;
    }
  } else {
    if (a.col_active != nullptr && a.col_active[col] == 0) return;  // uniform over the cluster
    member = a.col_member ? a.col_member[col] : col;
    voff = (long long)col * (a.mode == MODE_NL ? a.x0_stride : a.out_stride);
    soff = (long long)(a.mode == MODE_RHS ? member : col) * a.stash_stride;
    if (a.mode == MODE_NL) soff = (long long)col * a.p;
  }

  g.n = a.n;
  g.E = a.E;
  g.A = A_act;
  g.AS = blockDim.x;
  g.NT = blockDim.x;
  g.tid = threadIdx.x;
  g.tl = (g.tid + g.A - 1) % g.A;
  g.tr = (g.tid + 1) % g.A;
  g.l0 = g.tid * C;
  g.HL = a.HL;
  g.Ttile = a.Ttile;
  g.a0 = g.rank * a.Ttile;
  g.Town = min(a.Ttile, a.n - g.a0);
  g.gbase = ((g.a0 - a.HL) % a.n + a.n) % a.n;
  if (a.items == nullptr && a.mode != MODE_NL && bad_member(a, member)) {
    nan_owned(a, g, col, voff);  // uniform over the cluster: depends on col only
    return;
  }

  const int w = a.w;
  const int N = a.N;
  // shared memory: mirror | stage area (conv input, then edge buffers) | taps | obs map
  const int stage_sz = max(Emax + 2 * wmax + 2, kNumEdge * 4 * g.AS);
  T* mir = sm;
  T* stage = sm + Emax;
  T* eb[kNumEdge];
#pragma unroll
  for (int i = 0; i < kNumEdge; ++i) eb[i] = stage + i * 4 * g.AS;
  T* cf = stage + stage_sz;
  int* omap = reinterpret_cast<int*>(cf + (wmax + 1));
  const bool omap_smem = (N + 1) <= kObsMapCap;
  for (int j = g.tid; j <= w; j += g.NT) cf[j] = a.bcoef[j];
  if (omap_smem)
    for (int j = g.tid; j <= N; j += g.NT) omap[j] = a.obs_of_t[j];
  auto obs_at = [&](int t) { return omap_smem ? omap[t] : a.obs_of_t[t]; };
  // this CTA's rows of the observation range table, in shared memory when
  // they fit (every gather and injection reads them)
  const int* tabp = nullptr;
  if (a.obs_tab != nullptr) {
    const int* rows = a.obs_tab + (long long)g.rank * a.nos * 8;
    tabp = rows;
    if (a.nos * 8 <= kObsTabCap) {
      int* ot = omap + kObsMapCap;
      for (int j = g.tid; j < a.nos * 8; j += g.NT) ot[j] = rows[j];
      tabp = ot;
    }
  }

  // global indices of this thread's run, and whether vector loads apply (16
  // bytes, or 8 for a run of two FP32 values)
  int gi[C];
  {
    const int g0 = (g.gbase + g.l0) % g.n;
#pragma unroll
    for (int c = 0; c < C; ++c) gi[c] = (g0 + c) % g.n;
  }
  constexpr int kVec = (C * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : C;
  const bool vec_ok = (g.n % kVec == 0) && (gi[0] % kVec == 0) && (gi[0] + C <= g.n);

  const T F = a.F, h = a.dt;
  const T h2 = h * T(0.5), h6 = h / T(6), h3 = h / T(3);
  const bool clus = a.CS > 1 && !a.ml;
  const int f0 = a.ml ? a.f0 : 0, f1 = a.ml ? a.f1 : N;
  const int b0 = a.ml ? a.b0 : 0, b1 = a.ml ? a.b1 : N;
  // owned tile of a register run -> row[a0 .. a0 + Town) (through the mirror)
  auto store_owned = [&](const T (&v)[C], T* row) {
    write_mirror(mir, g, v);
    __syncthreads();
    for (int j = g.tid; j < g.Town; j += g.NT) row[g.a0 + j] = mir[g.HL + j];
    __syncthreads();
  };
  __syncthreads();

  if (a.mode == MODE_NL) {
    // ---------------------------------------------------------------- nonlinear
    T x[C];
    T* tout = a.traj_out ? a.traj_out + (long long)member * a.traj_out_mstride : nullptr;
    {
      // x_f0: the initial state, or (later launches of a multi-launch sweep)
      // the state the previous launch stored in the trajectory
      const T* x0row = (f0 == 0)        ? a.x0 + voff
                       : (tout != nullptr) ? tout + (long long)(a.ckpt ? f0 / a.ckpt : f0) * a.n
                                           : a.st_in + (long long)col * a.n;
      const bool x0_vec =
          vec_ok && ((reinterpret_cast<unsigned long long>(x0row) & (unsigned long long)(kVec * sizeof(T) - 1)) == 0);
      load_run<T, C>(x0row, gi, x0_vec, x);
    }
    // owned positions of a run -> row of a stage array
    T* sout = a.stage_out ? a.stage_out + (long long)member * a.traj_mstride : nullptr;
    auto store_stage = [&](int s_, int row, const T (&v)[C]) {
      T* dst = sout + (long long)s_ * a.stage_astride + (long long)row * a.n;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int l = g.l0 + c;
        if (l >= g.HL && l < g.HL + g.Town) dst[gi[c]] = v[c];
      }
    };
    // D_j = X_{j+1} - X_{j-2} of a stage state (its run with halos) -> array s_
    auto store_diff = [&](int s_, int row, const Run<T, C>& X) {
      T d[C];
#pragma unroll
      for (int c = 0; c < C; ++c) d[c] = X.at(c + 1) - X.at(c - 2);
      store_stage(s_, row, d);
    };
    for (int t = f0; t <= f1; ++t) {
      if (t > f0) {
        Run<T, C> X;
        T X1[C], acc[C], Xs[C];
#pragma unroll
        for (int c = 0; c < C; ++c) X1[c] = x[c];
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = x[c];
        fetch(eb[0], g, X);
        if (sout) store_diff(3, t - 1, X);  // D of X1 = x_t
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] = k;
          Xs[c] = X1[c] + h2 * k;
        }
        if (sout) store_stage(0, t - 1, Xs);
        publish(eb[1], g, Xs);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = Xs[c];
        fetch(eb[1], g, X);
        if (sout) store_diff(4, t - 1, X);  // D of X2
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] += T(2) * k;
          Xs[c] = X1[c] + h2 * k;
        }
        if (sout) store_stage(1, t - 1, Xs);
        publish(eb[2], g, Xs);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = Xs[c];
        fetch(eb[2], g, X);
        if (sout) store_diff(5, t - 1, X);  // D of X3
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] += T(2) * k;
          Xs[c] = X1[c] + h * k;
        }
        if (sout) store_stage(2, t - 1, Xs);
        publish(eb[1], g, Xs);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = Xs[c];
        fetch(eb[1], g, X);
        if (sout) store_diff(6, t - 1, X);  // D of X4
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] += k;
          x[c] = X1[c] + h6 * acc[c];
        }
      }
      const bool fresh = (t > f0) || (f0 == 0);  // x_t not yet stored / observed
      const int oj = fresh ? obs_at(t) : -1;
      const bool refresh = (t > 0) && (t % a.K == 0) && (t < N);
      // a checkpointed store keeps the rows t = j * ckpt only
      const bool trow = tout != nullptr && (a.ckpt == 0 || t % a.ckpt == 0);
      const bool store = fresh && (trow || (t == N && a.final_out != nullptr));
      if (oj >= 0 || refresh || store) {
        write_mirror(mir, g, x);
        sync_cluster_or_block(refresh && clus);
        if (trow) {
          T* dst = tout + (long long)(a.ckpt ? t / a.ckpt : t) * a.n + g.a0;
          for (int j = g.tid; j < g.Town; j += g.NT) dst[j] = mir[g.HL + j];
        }
        if (t == N && a.final_out != nullptr) {
          T* dst = a.final_out + voff + g.a0;
          for (int j = g.tid; j < g.Town; j += g.NT) dst[j] = mir[g.HL + j];
        }
        if (oj >= 0) {
          int k0, k1;
          if (tabp != nullptr) {
            const int* tb = obs_ranges(tabp, oj);
            k0 = tb[0];
            k1 = tb[1];
          } else {
            k0 = a.obs_ptr[oj];
            k1 = a.obs_ptr[oj + 1];
          }
          for (int k = k0 + g.tid; k < k1; k += g.NT) {
            const int gk = a.obs_idx[k];
            if (gk >= g.a0 && gk < g.a0 + g.Town) {
              const T hx = mir[g.HL + gk - g.a0];
              const T d = a.yobs ? a.yobs[soff + k] - hx : hx;
              if (a.d_out) a.d_out[soff + k] = d;
              if (a.rd_out) a.rd_out[soff + k] = a.rinv[k] * d;
            }
          }
        }
        if (refresh) {
          read_halo(x, mir, g);
          sync_cluster_or_block(clus);
        }
      }
      publish(eb[0], g, x);
      __syncthreads();
    }
    if (a.ml && tout == nullptr && f1 < N) store_owned(x, a.st_out + (long long)col * a.n);
    return;
  }

  // ------------------------------------------------------------------ HVP / RHS
  const T* trj = a.traj + (long long)member * a.traj_mstride;
  const T* V = (a.mode == MODE_HVP && a.V) ? a.V + voff : nullptr;
  const double* V64 = (a.mode == MODE_HVP && a.V64) ? a.V64 + voff : nullptr;
  T* stash = a.stash + soff;
  T xr[C];  // own run of x_t (registers)
  // stored stage states of this member (or recomputation when absent)
  const T* stg = nullptr;
  if constexpr (STG) stg = a.stages ? a.stages + (long long)member * a.traj_mstride : nullptr;
  int gh[4];  // global indices of the run's two left and two right neighbours
  gh[0] = (gi[0] - 2 + g.n) % g.n;
  gh[1] = (gi[0] - 1 + g.n) % g.n;
  gh[2] = (gi[C - 1] + 1) % g.n;
  gh[3] = (gi[C - 1] + 2) % g.n;
  auto load_halo = [&](const T* row, Run<T, C>& X) {
    X.m2 = row[gh[0]];
    X.m1 = row[gh[1]];
    X.p1 = row[gh[2]];
    X.p2 = row[gh[3]];
  };
  auto load_sx = [&](const T* row, Run<T, C>& X) {
    load_run<T, C>(row, gi, vec_ok, X.v);
    load_halo(row, X);
  };
  // checkpointed trajectory: the states of this launch's steps, recomputed
  // from the segment's checkpoint over the extended region into shared
  // memory (rows seg0 .. seg0 + cnt - 1); their edge errors are covered by
  // the plan's wider halo
  T* xseg = (CK && a.ckpt) ? reinterpret_cast<T*>(smem_raw + a.xseg_off) : nullptr;
  int seg0 = 0;
  auto recompute = [&](int s0, int cnt) {
    seg0 = s0;
    T x[C];
    load_run<T, C>(trj + (long long)(s0 / a.ckpt) * a.n, gi, vec_ok, x);
    for (int s_ = 0; s_ < cnt; ++s_) {
      if (s_ > 0) {  // one RK4 step of the model, as the nonlinear sweep takes it
        publish(eb[0], g, x);
        __syncthreads();
        Run<T, C> X;
        T X1[C], acc[C], Xs[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          X1[c] = x[c];
          X.v[c] = x[c];
        }
        fetch(eb[0], g, X);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] = k;
          Xs[c] = X1[c] + h2 * k;
        }
        publish(eb[1], g, Xs);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = Xs[c];
        fetch(eb[1], g, X);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] += T(2) * k;
          Xs[c] = X1[c] + h2 * k;
        }
        publish(eb[2], g, Xs);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = Xs[c];
        fetch(eb[2], g, X);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] += T(2) * k;
          Xs[c] = X1[c] + h * k;
        }
        publish(eb[1], g, Xs);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) X.v[c] = Xs[c];
        fetch(eb[1], g, X);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T k = tend(X, c, F);
          acc[c] += k;
          x[c] = X1[c] + h6 * acc[c];
        }
      }
      write_mirror(xseg + (long long)s_ * g.E, g, x);
    }
    __syncthreads();
  };
  // own run of x_t: the recomputed segment, or the stored trajectory
  auto xrow = [&](int t, T (&out)[C]) {
    if constexpr (CK) {
      if (xseg != nullptr) {
        const T* src = xseg + (long long)(t - seg0) * g.E + g.l0;
#pragma unroll
        for (int c = 0; c < C; ++c) out[c] = src[c];
        return;
      }
    }
    load_run<T, C>(trj + (long long)t * a.n, gi, vec_ok, out);
  };

  if (a.mode == MODE_HVP && f1 > f0) {
    T dl[C];
    if constexpr (CK) {
      if (xseg != nullptr) recompute(f0, f1 - f0);
    }
    if (f0 == 0) {
    // delta_0 = U_B v on the extended region (v staged with a w-halo)
    {
      const int cnt = g.E + 2 * w;
      for (int j = g.tid; j < cnt; j += g.NT) {
        int gk = (g.gbase - w + j) % g.n;
        if (gk < 0) gk += g.n;
        stage[j] = V64 ? (T)__ldcg(V64 + gk) : __ldcg(V + gk);
      }
      __syncthreads();
    }
    conv_run<T, C>(stage, g.l0, w, cf, dl);
    xrow(0, xr);
    __syncthreads();  // the stage area becomes the edge buffers
    if (obs_at(0) >= 0) {
      write_mirror(mir, g, dl);
      __syncthreads();
      gather_obs(a, g, obs_at(0), tabp, mir, stash);
    }
    } else {
      // later launch of a multi-launch sweep: the state of the extended region
      load_run<T, C>(a.st_in + (long long)col * a.n, gi, vec_ok, dl);
      xrow(f0, xr);
    }
    publish(eb[0], g, dl);
    publish(eb[5], g, xr);
    __syncthreads();

    // ------------------------------------------------ tangent linear, forward
    // FP32 sweeps of four values per thread load the observations of
    // x_{t+1} at the start of step t (the other instantiations keep their
    // registers for the stages)
    constexpr bool kPre = sizeof(T) == 4 && C == 4;
    for (int t = f0; t < f1; ++t) {
      T pf[C];
      if (t + 1 < f1) xrow(t + 1, pf);
      int oj_pre = -1;
      ObsPre<T> qg;
      if constexpr (kPre) {
        oj_pre = obs_at(t + 1);
        if (oj_pre >= 0 && tabp != nullptr) gather_pre(a, g, obs_ranges(tabp, oj_pre), qg);
      }
      if (stg != nullptr) {
        // stage states X_s and their differences D_s from the store (arrays
        // 0-2: X2..X4, 3-6: D of X1..X4): each slope is three FP64
        // instructions (jvpd); only delta's edges are exchanged
        T xm[4][C], dd[4][C];  // X_s[j-1] and D_s[j] over the run
        {
          const T* r1 = trj + (long long)t * a.n;
          xm[0][0] = r1[gh[1]];
#pragma unroll
          for (int c = 1; c < C; ++c) xm[0][c] = xr[c - 1];
#pragma unroll
          for (int s_ = 1; s_ < 4; ++s_) {
            const T* row = stg + (long long)(s_ - 1) * a.stage_astride + (long long)t * a.n;
            T v[C];
            load_run<T, C>(row, gi, vec_ok, v);
            xm[s_][0] = row[gh[1]];
#pragma unroll
            for (int c = 1; c < C; ++c) xm[s_][c] = v[c - 1];
          }
#pragma unroll
          for (int s_ = 0; s_ < 4; ++s_)
            load_run<T, C>(stg + (long long)(3 + s_) * a.stage_astride + (long long)t * a.n, gi, vec_ok, dd[s_]);
        }
        Run<T, C> e;
        T es[C], acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) e.v[c] = dl[c];
        fetch(eb[0], g, e);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T dk = jvpd(xm[0][c], dd[0][c], e, c);
          acc[c] = dk;
          es[c] = fma(h2, dk, dl[c]);
        }
        publish(eb[3], g, es);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) e.v[c] = es[c];
        fetch(eb[3], g, e);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T dk = jvpd(xm[1][c], dd[1][c], e, c);
          acc[c] = fma(T(2), dk, acc[c]);
          es[c] = fma(h2, dk, dl[c]);
        }
        publish(eb[4], g, es);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) e.v[c] = es[c];
        fetch(eb[4], g, e);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T dk = jvpd(xm[2][c], dd[2][c], e, c);
          acc[c] = fma(T(2), dk, acc[c]);
          es[c] = fma(h, dk, dl[c]);
        }
        publish(eb[3], g, es);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) e.v[c] = es[c];
        fetch(eb[3], g, e);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          acc[c] += jvpd(xm[3][c], dd[3][c], e, c);
          dl[c] = fma(h6, acc[c], dl[c]);
        }
      } else {
      Run<T, C> X, e;
      T Xs[C], es[C], acc[C];
      // stage 1: slopes at X1 = x_t
#pragma unroll
      for (int c = 0; c < C; ++c) {
        X.v[c] = xr[c];
        e.v[c] = dl[c];
      }
      fetch(eb[5], g, X);
      fetch(eb[0], g, e);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T k = tend(X, c, F);
        const T dk = jvp(X, e, c);
        Xs[c] = xr[c] + h2 * k;
        acc[c] = dk;
        es[c] = dl[c] + h2 * dk;
      }
      publish(eb[1], g, Xs);
      publish(eb[3], g, es);
      __syncthreads();
      // stage 2
#pragma unroll
      for (int c = 0; c < C; ++c) {
        X.v[c] = Xs[c];
        e.v[c] = es[c];
      }
      fetch(eb[1], g, X);
      fetch(eb[3], g, e);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T k = tend(X, c, F);
        const T dk = jvp(X, e, c);
        Xs[c] = xr[c] + h2 * k;
        acc[c] += T(2) * dk;
        es[c] = dl[c] + h2 * dk;
      }
      publish(eb[2], g, Xs);
      publish(eb[4], g, es);
      __syncthreads();
      // stage 3
#pragma unroll
      for (int c = 0; c < C; ++c) {
        X.v[c] = Xs[c];
        e.v[c] = es[c];
      }
      fetch(eb[2], g, X);
      fetch(eb[4], g, e);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T k = tend(X, c, F);
        const T dk = jvp(X, e, c);
        Xs[c] = xr[c] + h * k;
        acc[c] += T(2) * dk;
        es[c] = dl[c] + h * dk;
      }
      publish(eb[1], g, Xs);
      publish(eb[3], g, es);
      __syncthreads();
      // stage 4
#pragma unroll
      for (int c = 0; c < C; ++c) {
        X.v[c] = Xs[c];
        e.v[c] = es[c];
      }
      fetch(eb[1], g, X);
      fetch(eb[3], g, e);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T dk = jvp(X, e, c);
        acc[c] += dk;
        dl[c] += h6 * acc[c];
      }
      }
      if (t + 1 < f1) {
#pragma unroll
        for (int c = 0; c < C; ++c) xr[c] = pf[c];
      }
      const int oj = kPre ? oj_pre : obs_at(t + 1);
      const bool refresh = ((t + 1) % a.K == 0) && (t + 1 < N);
      if (oj >= 0 || refresh) {
        write_mirror(mir, g, dl);
        sync_cluster_or_block(refresh && clus);
        if (oj >= 0) {
          if (kPre && tabp != nullptr)
            gather_use(a, g, obs_ranges(tabp, oj), qg, mir, stash);
          else
            gather_obs(a, g, oj, tabp, mir, stash);
        }
        if (refresh) {
          read_halo(dl, mir, g);
          sync_cluster_or_block(clus);
        }
      }
      publish(eb[0], g, dl);
      publish(eb[5], g, xr);
      __syncthreads();
    }
    // the stash written by every CTA of the cluster must be visible to all
    if (clus) cg::this_cluster().sync();
    if (a.ml && f1 < N) store_owned(dl, a.st_out + (long long)col * a.n);
  }
  if (b1 <= b0) return;  // a forward-only launch of a multi-launch sweep

  // ------------------------------------------------------ adjoint, backward
  if constexpr (CK) {
    if (xseg != nullptr) recompute(b0, b1 - b0);
  }
  T lam[C];
#pragma unroll
  for (int c = 0; c < C; ++c) lam[c] = T(0);

  auto inject = [&](int oj, const ObsPre<T>* q) {
    write_mirror_zero<T, C>(mir, g);
    __syncthreads();
    if (q != nullptr) {
      inject_use(a, g, obs_ranges(tabp, oj), *q, stash, mir);
    } else if (tabp != nullptr) {
      const int* tb = obs_ranges(tabp, oj);
#pragma unroll
      for (int sgm = 0; sgm < 2; ++sgm) {
        const int k0 = tb[2 + 3 * sgm], k1 = tb[3 + 3 * sgm], base = tb[4 + 3 * sgm];
        scatter_obs<T>(a.obs_idx, stash, k0, k1, base, g.tid, g.NT, mir);
      }
    } else {
      const int k0 = a.obs_ptr[oj], k1 = a.obs_ptr[oj + 1];
      for (int k = k0 + g.tid; k < k1; k += g.NT) {
        const int gk = a.obs_idx[k];
        const T val = __ldcg(stash + k);
        int l = ((gk - g.gbase) % g.n + g.n) % g.n;
        for (; l < g.E; l += g.n) mir[l] = val;
      }
    }
    __syncthreads();
    add_mirror<T, C>(mir, g, lam);
  };

  if (b1 == N) {
    if (obs_at(N) >= 0) inject(obs_at(N), nullptr);
  } else {
    load_run<T, C>(a.st_in + (long long)col * a.n, gi, vec_ok, lam);
  }
  xrow(b1 - 1, xr);
  publish(eb[0], g, xr);
  __syncthreads();
  // FP32 sweeps of four values per thread load the injection of step t at
  // its start
  constexpr bool kPreA = sizeof(T) == 4 && C == 4;
  for (int t = b1 - 1; t >= b0; --t) {
    T pf[C];
    if (t > b0) xrow(t - 1, pf);
    int oj_pre = -1;
    ObsPre<T> qa;
    if constexpr (kPreA) {
      oj_pre = obs_at(t);
      if (oj_pre >= 0 && tabp != nullptr) inject_pre(a, g, obs_ranges(tabp, oj_pre), stash, qa);
    }
    if (stg != nullptr) {
      // stage states and their differences from the store (jtvpd: three
      // FP64 instructions per slope); only the adjoint weights' edges are
      // exchanged, through edge buffers 3 and 4 in turn
      Run<T, C> S[4], wv;
      T dp[4][C];  // D_s[j+1] over the run
      T ln[C], ad[C];
      {
        const T* r1 = trj + (long long)t * a.n;
#pragma unroll
        for (int c = 0; c < C; ++c) S[0].v[c] = xr[c];
        S[0].m2 = r1[gh[0]];
        S[0].m1 = r1[gh[1]];
        S[0].p1 = r1[gh[2]];
#pragma unroll
        for (int s_ = 1; s_ < 4; ++s_) {
          const T* row = stg + (long long)(s_ - 1) * a.stage_astride + (long long)t * a.n;
          load_run<T, C>(row, gi, vec_ok, S[s_].v);
          S[s_].m2 = row[gh[0]];
          S[s_].m1 = row[gh[1]];
          S[s_].p1 = row[gh[2]];
        }
#pragma unroll
        for (int s_ = 0; s_ < 4; ++s_) {
          const T* row = stg + (long long)(3 + s_) * a.stage_astride + (long long)t * a.n;
          T v[C];
          load_run<T, C>(row, gi, vec_ok, v);
#pragma unroll
          for (int c = 0; c + 1 < C; ++c) dp[s_][c] = v[c + 1];
          dp[s_][C - 1] = row[gh[2]];
        }
      }
      // the reverse RK4 step (u_s = J_s^T b_s, b4 = lam) on the stored stages
#pragma unroll
      for (int c = 0; c < C; ++c) wv.v[c] = lam[c];
      publish(eb[3], g, lam);
      __syncthreads();
      fetch(eb[3], g, wv);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T u = jtvpd(S[3], dp[3][c], wv, c);
        ln[c] = fma(h6, u, lam[c]);
        ad[c] = fma(h2, u, lam[c]);  // b3
      }
      publish(eb[4], g, ad);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
      fetch(eb[4], g, wv);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T u = jtvpd(S[2], dp[2][c], wv, c);
        ln[c] = fma(h3, u, ln[c]);
        ad[c] = fma(h2, u, lam[c]);  // b2
      }
      publish(eb[3], g, ad);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
      fetch(eb[3], g, wv);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T u = jtvpd(S[1], dp[1][c], wv, c);
        ln[c] = fma(h3, u, ln[c]);
        ad[c] = fma(h, u, lam[c]);  // b1
      }
      publish(eb[4], g, ad);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
      fetch(eb[4], g, wv);
#pragma unroll
      for (int c = 0; c < C; ++c) lam[c] = fma(h6, jtvpd(S[0], dp[0][c], wv, c), ln[c]);
    } else {
    Run<T, C> X1, X, wv;
    T X2[C], X3[C], X4[C], ln[C], ad[C];
    // forward recomputation of the stage states
#pragma unroll
    for (int c = 0; c < C; ++c) X1.v[c] = xr[c];
    fetch(eb[0], g, X1);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X2[c] = xr[c] + h2 * tend(X1, c, F);
      ad[c] = lam[c];  // b4
    }
    publish(eb[1], g, X2);
    publish(eb[3], g, ad);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) X.v[c] = X2[c];
    fetch(eb[1], g, X);
#pragma unroll
    for (int c = 0; c < C; ++c) X3[c] = xr[c] + h2 * tend(X, c, F);
    publish(eb[2], g, X3);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) X.v[c] = X3[c];
    fetch(eb[2], g, X);
#pragma unroll
    for (int c = 0; c < C; ++c) X4[c] = xr[c] + h * tend(X, c, F);
    publish(eb[5], g, X4);
    __syncthreads();
    // reverse stage 4: u4 = J4^T b4, b4 = lam (the reverse RK4 step)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = X4[c];
      wv.v[c] = ad[c];
    }
    fetch(eb[5], g, X);
    fetch(eb[3], g, wv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T u = jtvp(X, wv, c);
      ln[c] = fma(h6, u, lam[c]);
      ad[c] = fma(h2, u, lam[c]);  // b3
    }
    publish(eb[4], g, ad);
    __syncthreads();
    // reverse stage 3
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = X3[c];
      wv.v[c] = ad[c];
    }
    fetch(eb[2], g, X);
    fetch(eb[4], g, wv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T u = jtvp(X, wv, c);
      ln[c] = fma(h3, u, ln[c]);
      ad[c] = fma(h2, u, lam[c]);  // b2
    }
    publish(eb[3], g, ad);
    __syncthreads();
    // reverse stage 2
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = X2[c];
      wv.v[c] = ad[c];
    }
    fetch(eb[1], g, X);
    fetch(eb[3], g, wv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T u = jtvp(X, wv, c);
      ln[c] = fma(h3, u, ln[c]);
      ad[c] = fma(h, u, lam[c]);  // b1
    }
    publish(eb[4], g, ad);
    __syncthreads();
    // reverse stage 1
#pragma unroll
    for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
    fetch(eb[4], g, wv);
#pragma unroll
    for (int c = 0; c < C; ++c) lam[c] = fma(h6, jtvp(X1, wv, c), ln[c]);
    }
    if (t > b0) {
#pragma unroll
      for (int c = 0; c < C; ++c) xr[c] = pf[c];
    }
    const int oj = kPreA ? oj_pre : obs_at(t);
    if (oj >= 0) {
      if constexpr (kPreA)
        inject(oj, tabp != nullptr ? &qa : nullptr);
      else
        inject(oj, nullptr);
    }
    const bool refresh = ((N - t) % a.K == 0) && (t > 0);
    if (refresh) {
      write_mirror(mir, g, lam);
      sync_cluster_or_block(clus);
      read_halo(lam, mir, g);
      sync_cluster_or_block(clus);
    }
    if (stg == nullptr) {  // the recomputation reads x_t's edges from buffer 0
      publish(eb[0], g, xr);
      __syncthreads();
    }
  }

  if (a.ml) {  // multi-launch: the state goes to global memory; U_B follows in its own kernel
    store_owned(lam, a.st_out + (long long)col * a.n);
    return;
  }
  // ---------------------------------------------- output U_B lambda_0 (+ v)
  write_mirror(mir, g, lam);
  sync_cluster_or_block(clus);
  const bool ident = (a.mode == MODE_HVP && a.include_identity);
  double* dot = (ident && a.dot_out != nullptr) ? a.dot_out + (long long)item * a.dot_stride : nullptr;
  if (a.OUT64) {
    bhalf_from_mirrors<T, C, double>(a, g, mir, stage, cf, a.OUT64 + voff, ident ? V64 : nullptr,
                                     ident ? V : nullptr, dot);
  } else {
    bhalf_from_mirrors<T, C, T>(a, g, mir, stage, cf, a.OUT + voff, ident ? V64 : nullptr, ident ? V : nullptr,
                                dot);
  }
}

template <typename T, int C, bool STG, bool CK>
__global__ void __launch_bounds__(kMaxThreads) sweep_kernel(const SweepArgs<T> a0) {
  sweep_body<T, C, STG, CK>(a0, (int)(blockIdx.x / a0.CS));
}

// Sum of v over the CTA (every thread gets it); red: 32 doubles of shared
// memory that no other code uses in between.
__device__ __forceinline__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// Persistent PCG (pcg.h): one member's whole PCG loop run by this cluster.
// Every decision to leave the loop is taken by every CTA of the cluster from
// the same values (read after the same cluster barrier), so the cluster's
// barriers stay matched; every member stops by its iteration budget at the
// latest.  Values other CTAs write during the launch (the accumulators, the
// projections, p's halo in the sweep) are read past L1 (__ldcg).
//   scol  the member's column for the sweep (index into sw.items in group
//         mode); j its PCG index; n its state size; Ttile the tile of this
//         plan; voff the offset of its vectors; S, cvec, k its LMP.
template <typename T, int C, bool STG>
__device__ __forceinline__ void persist_member(const PersistArgs<T>& P, SweepArgs<T>& a, int scol, int j, int n,
                                               int Ttile, long long voff, const T* S, const double* cvec, int k,
                                               int rank) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CS = P.sw.CS, kmax = P.kmax;
  const int a0 = rank * Ttile;
  const int town = min(Ttile, n - a0);
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = NT >> 5;
  const long long vo = voff + a0;
  // scratch between sweeps (the sweep re-initialises its shared memory)
  double* red = reinterpret_cast<double*>(smem_raw);
  T* cw = reinterpret_cast<T*>(red + 32);
  T* rt = cw + ((kmax + 3) & ~3);
  PersistAcc* pa = P.pacc + j;
  T* Wj[2] = {P.W + (long long)j * kmax, P.W + ((long long)P.M + j) * kmax};
  auto csync = [&]() {
    __threadfence();
    if (CS > 1) cg::this_cluster().sync();
    else __syncthreads();
  };
  double rz = __ldcg(&P.acc[j].rz[0]);
  int it = P.sc[j].iters;
  const double bn = P.sc[j].bnorm;
  const double tolm = P.sc[j].tolm;
  double rel = P.sc[j].relres;
  int status = EDA_MAXIT;
  int par = 0;
  a.dot_stride = (int)(sizeof(PersistAcc) / sizeof(double));
  for (;;) {
    // q = (I + A) p with p.q into this iteration's slot
    a.dot_out = &P.pacc[0].pq[par];
    sweep_body<T, C, STG, false>(a, scol);
    csync();
    const double pq = __ldcg(&pa->pq[par]);
    if (!(pq > 0.0)) {  // breakdown (or NaN): uniform
      status = isfinite(pq) ? EDA_BREAKDOWN : EDA_NAN;
      break;
    }
    const double alpha = rz / pq;
    double rr = 0.0, xx = 0.0;
    for (int i = tid; i < town; i += NT) {
      const long long g = vo + i;
      const double xn = P.x[g] + alpha * P.p[g];
      const double rn = P.r[g] - alpha * P.q[g];
      P.x[g] = xn;
      P.r[g] = rn;
      rr += rn * rn;
      xx += xn * xn;
      rt[i] = (T)rn;
    }
    __syncthreads();
    // the LMP projections of the new r over this tile: warp w takes modes
    // w, w + nw, ...
    for (int c = wid; c < k; c += nw) {
      const T* Sc = S + (long long)c * n + a0;
      T s0 = T(0);
      for (int i = lane; i < town; i += 32) s0 += Sc[i] * rt[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      if (lane == 0) atomicAdd(&Wj[par][c], s0);
    }
    rr = cta_sum(rr, red);
    xx = cta_sum(xx, red);
    if (tid == 0) {
      atomicAdd(&pa->rr[par], rr);
      atomicAdd(&pa->xx[par], xx);
    }
    csync();
    const double rrt = __ldcg(&pa->rr[par]), xxt = __ldcg(&pa->xx[par]);
    ++it;
    // the stopping test of pcg2_precond
    rel = bn > 0.0 ? sqrt(rrt) / bn : 0.0;
    bool stop = false;
    if (!isfinite(rel)) {
      status = EDA_NAN;
      stop = true;
    } else if (P.fixed > 0) {
      if (it >= P.fixed) {
        status = EDA_CONVERGED;
        stop = true;
      }
    } else {
      bool fin = !(P.tol > 0.0) || rel <= P.tol;
      if (P.etol > 0.0) {
        const double rn = rel * bn, xn = sqrt(xxt);
        fin = fin && xn > rn && rn <= P.etol * (xn - rn);
      }
      if (fin || (tolm > 0.0 && rel <= tolm)) {
        status = EDA_CONVERGED;
        stop = true;
      } else if (it >= P.maxit) {  // the host launches this loop with maxit >= 1
        status = EDA_MAXIT;
        stop = true;
      }
    }
    if (stop) break;
    // z = r + S (c o w), r.z
    for (int c = tid; c < k; c += NT) cw[c] = (T)(cvec[c] * (double)__ldcg(&Wj[par][c]));
    __syncthreads();
    double rzp = 0.0;
    for (int i = tid; i < town; i += NT) {
      const long long g = vo + i;
      T s0 = T(0), s1 = T(0);
      int c = 0;
      for (; c + 2 <= k; c += 2) {
        s0 += S[(long long)c * n + a0 + i] * cw[c];
        s1 += S[(long long)(c + 1) * n + a0 + i] * cw[c + 1];
      }
      if (c < k) s0 += S[(long long)c * n + a0 + i] * cw[c];
      const double rv = P.r[g];
      const double zv = rv + (double)(s0 + s1);
      P.z[g] = zv;
      rzp += rv * zv;
    }
    rzp = cta_sum(rzp, red);
    if (tid == 0) atomicAdd(&pa->rz[par], rzp);
    csync();
    const double rzn = __ldcg(&pa->rz[par]);
    const double beta = rzn / rz;
    rz = rzn;
    for (int i = tid; i < town; i += NT) {
      const long long g = vo + i;
      P.p[g] = P.z[g] + beta * P.p[g];
    }
    // the other parity's slots were read last iteration: clear them for the next
    if (rank == 0) {
      if (tid == 0) {
        pa->pq[par ^ 1] = 0.0;
        pa->rr[par ^ 1] = 0.0;
        pa->xx[par ^ 1] = 0.0;
        pa->rz[par ^ 1] = 0.0;
        // the launch's exit flag, published for the whole cluster (ex[par]
        // was last read two barriers ago)
        if (P.brk != nullptr) pa->ex[par] = *reinterpret_cast<volatile int*>(P.brk) != 0 ? 1.0 : 0.0;
      }
      for (int c = tid; c < k; c += NT) Wj[par ^ 1][c] = T(0);
    }
    csync();  // p complete (the next sweep reads its halo) and the slots cleared
    if (P.brk != nullptr && __ldcg(&pa->ex[par]) != 0.0) {  // uniform: read after the same barrier
      // leave with the state of a completed iteration: the next launch
      // starts with the sweep of this p and reads r.z from acc[j].rz[0]
      if (rank == 0 && tid == 0) {
        P.sc[j].iters = it;
        P.sc[j].relres = rel;
        P.acc[j].rz[0] = rz;
      }
      return;
    }
    par ^= 1;
  }
  if (rank == 0 && tid == 0) {
    P.sc[j].iters = it;
    P.sc[j].status = status;
    P.sc[j].relres = rel;
    P.active[j] = 0;
    const int left = atomicSub(P.nactive, 1) - 1;
    if (P.brk != nullptr && left <= P.exit_below) atomicExch(P.brk, 1);
  }
}

// One member per cluster (a handle's solve), or, in group mode (GROUP), the
// members of the launch's items taken in turn from the device-side queue.
template <typename T, int C, bool STG, bool GROUP>
__global__ void __launch_bounds__(kMaxThreads) pcg_persist_kernel(const PersistArgs<T> P) {
  __shared__ int next_item;
  const int CS = P.sw.CS;
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  SweepArgs<T> a = P.sw;
  if constexpr (!GROUP) {
    const int col = (int)blockIdx.x / CS;
    if (col >= P.M) return;          // uniform over the cluster
    if (P.active[col] == 0) return;  // uniform: written before the launch
    persist_member<T, C, STG>(P, a, col, col, P.n, P.sw.Ttile, (long long)col * P.n, P.S, P.c,
                              P.use_lmp ? P.k : 0, rank);
    return;
  } else {
  for (;;) {
    // rank 0 takes the next item for the cluster; the others read it from
    // rank 0's shared memory between two cluster barriers
    if (rank == 0 && threadIdx.x == 0) next_item = atomicAdd(P.queue, 1);
    int idx;
    if (CS > 1) {
      cg::this_cluster().sync();
      idx = *cg::this_cluster().map_shared_rank(&next_item, 0);
      cg::this_cluster().sync();
    } else {
      __syncthreads();
      idx = next_item;
      __syncthreads();
    }
    if (idx >= P.nitems) return;  // uniform: every CTA read the same index
    const SweepItem itm = P.items[idx];
    const int j = itm.flag;
    if (j < 0 || P.active[j] == 0) continue;  // uniform
    const PcgProb pp = P.pprobs[itm.prob];
    const SweepProb<T> sp = P.sw.probs[itm.prob];
    persist_member<T, C, STG>(P, a, idx, j, sp.n, sp.Ttile, itm.voff, static_cast<const T*>(pp.S), pp.c,
                              P.use_lmp ? pp.k : 0, rank);
  }
  }
}

template <typename T, int C, bool STG, bool GROUP = false>
cudaError_t launch_persist_impl(const PersistArgs<T>& a, const SweepPlan& p, cudaStream_t s, int* query) {
  auto kern = pcg_persist_kernel<T, C, STG, GROUP>;
  static bool attrs_set = false;
  if (!attrs_set) {
    // the group kernel's static shared memory (the queue slot) counts against the 227 KB
    cudaFuncAttributes fa{};
    cudaError_t err = cudaFuncGetAttributes(&fa, kern);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               227 * 1024 - (int)fa.sharedSizeBytes);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
    attrs_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.M * p.CS), 1, 1);
  cfg.blockDim = dim3((unsigned)p.A, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (p.CS > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  if (query != nullptr) {
    // how many of this launch's clusters fit on the device at once (0: none)
    *query = 0;
    if (p.CS > 1) {
      if (cudaOccupancyMaxActiveClusters(query, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        *query = 0;
      }
    } else {
      int dev = 0, sms = 0, per_sm = 0;
      if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                                    cudaSuccess &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.A, p.smem) == cudaSuccess)
        *query = per_sm * sms;
      else
        (void)cudaGetLastError();
    }
    return cudaSuccess;
  }
  if (a.items != nullptr) {
    // group mode: as many clusters as fit at once (they loop over the queue;
    // clusters beyond what fits wait and then find the queue empty)
    int dev = 0, sms = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.A, p.smem) != cudaSuccess || per_sm < 1) {
      (void)cudaGetLastError();
      per_sm = 1;
    }
    int clusters = 0;
    if (p.CS > 1) {
      if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        clusters = 0;
      }
    }
    if (clusters < 1) clusters = per_sm * sms / (p.CS > 0 ? p.CS : 1);
    if (clusters < 1) clusters = 1;
    if (clusters > a.nitems) clusters = a.nitems;
    cfg.gridDim = dim3((unsigned)(clusters * p.CS), 1, 1);
    const char* vb = std::getenv("EDA_VERBOSE");
    if (vb != nullptr && std::atoi(vb) != 0)
      std::fprintf(stderr, "persistent group launch: CS=%d A=%d smem=%zu items=%d clusters=%d\n", p.CS, p.A,
                   p.smem, a.nitems, clusters);
  }
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// out[col][i] = (ident ? v[col][i] : 0) + sum_{|d|<=w} coef[|d|] lam[col][(i+d) mod n]
// (the last step of a multi-launch Hessian product or right-hand side).
template <typename T, typename TO>
__global__ void bhalf_out_kernel(int n, int w, const T* __restrict__ coef, int ncol, const T* __restrict__ lam,
                                 const double* v64, const T* v, TO* out, int ident) {
  const long long total = (long long)ncol * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const T* row = lam + (e - i);
    T acc = coef[0] * row[i];
    for (int d = 1; d <= w; ++d) {
      int im = i - d;
      if (im < 0) im += n;
      int ip = i + d;
      if (ip >= n) ip -= n;
      acc += coef[d] * (row[im] + row[ip]);
    }
    TO o = (TO)acc;
    if (ident) o += v64 ? (TO)v64[e] : (TO)v[e];
    out[e] = o;
  }
}

// ---------------------------------------------------------------------------
// Warp-tiled Hessian-vector sweep (MODE_HVP).  As above, one column per
// cluster of CS CTAs, each CTA computing an extended region of E points with
// a halo of 8K + 8 refreshed from the owners every K steps.  Inside the CTA
// the region is split among warps: warp w owns E positions
// [w*LW, (w+1)*LW) and computes on the 32*C points starting HW before them
// (HW = warp_halo(C), LW = 32*C - 2*HW), lane l holding C consecutive
// values.  Stencil neighbours come from warp shuffles; one RK4 step spreads
// an edge error at most 11 points, so after every step each warp publishes
// its owned values to a shared mirror (double-buffered by step parity) and
// its edge lanes reload theirs after one block barrier.  Observation gather and
// injection touch only the warp's own positions, through a per-(rank, warp,
// observation step) table of index ranges.
// ---------------------------------------------------------------------------
// Positions a one-step error can travel from a tile edge: 8 (left) and 4
// (right) in a tangent-linear RK4 step, 11 both ways in an adjoint step with
// its stage recomputation.  A warp halo is the smallest whole number of runs
// covering 11 points.
__host__ __device__ constexpr int warp_halo(int C) { return ((11 + C - 1) / C) * C; }
constexpr int kWarpMaxThreads = 512;

template <typename T, int C>
__device__ __forceinline__ void shfl_m2m1p1(Run<T, C>& r) {
  r.m2 = __shfl_up_sync(0xffffffffu, r.v[C - 2], 1);
  r.m1 = __shfl_up_sync(0xffffffffu, r.v[C - 1], 1);
  r.p1 = __shfl_down_sync(0xffffffffu, r.v[0], 1);
}
template <typename T, int C>
__device__ __forceinline__ void shfl_all(Run<T, C>& r) {
  shfl_m2m1p1<T, C>(r);
  r.p2 = __shfl_down_sync(0xffffffffu, r.v[1], 1);
}
template <typename T, int C>
__device__ __forceinline__ void shfl_m1p1p2(Run<T, C>& r) {
  r.m1 = __shfl_up_sync(0xffffffffu, r.v[C - 1], 1);
  r.p1 = __shfl_down_sync(0xffffffffu, r.v[0], 1);
  r.p2 = __shfl_down_sync(0xffffffffu, r.v[1], 1);
}

template <typename T, int C>
__device__ __forceinline__ void run_to_smem(T* dst, const T (&v)[C]) {
  if constexpr (sizeof(T) == 4) {
    float4* q = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < C / 4; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    double2* q = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int i = 0; i < C / 2; ++i) q[i] = make_double2(v[2 * i], v[2 * i + 1]);
  }
}
template <typename T, int C>
__device__ __forceinline__ void run_from_smem_vec(const T* src, T (&v)[C]) {
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < C / 4; ++i) {
      const float4 u = q[i];
      v[4 * i] = u.x;
      v[4 * i + 1] = u.y;
      v[4 * i + 2] = u.z;
      v[4 * i + 3] = u.w;
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
      const double2 u = q[i];
      v[2 * i] = u.x;
      v[2 * i + 1] = u.y;
    }
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(kWarpMaxThreads) wsweep_kernel(const SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int HW = warp_halo(C);
  constexpr int HLN = HW / C;          // edge lanes on each side of a warp tile
  constexpr int LW = 32 * C - 2 * HW;  // positions a warp owns
  static_assert(HW % C == 0, "the warp halo must be whole runs");
  const int nw = (int)(blockDim.x >> 5);
  const int wid = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);

  Geo g;
  g.CS = a.CS;
  g.rank = (a.CS > 1) ? (int)cg::this_cluster().block_rank() : 0;
  const int col = blockIdx.x / a.CS;
  if (col >= a.ncol) return;
  if (a.col_active != nullptr && a.col_active[col] == 0) return;  // uniform over the cluster
  const int member = a.col_member ? a.col_member[col] : col;
  const long long voff = (long long)col * a.out_stride;
  const long long soff = (long long)col * a.stash_stride;
  g.n = a.n;
  g.E = a.E;
  g.A = g.AS = g.NT = (int)blockDim.x;
  g.tid = (int)threadIdx.x;
  g.tl = g.tr = g.l0 = 0;
  g.HL = a.HL;
  g.Ttile = a.Ttile;
  g.a0 = g.rank * a.Ttile;
  g.Town = min(a.Ttile, a.n - g.a0);
  g.gbase = ((g.a0 - a.HL) % a.n + a.n) % a.n;
  if (bad_member(a, member)) {
    nan_owned(a, g, col, voff);  // uniform over the cluster: depends on col only
    return;
  }
  const int E = a.E, w = a.w, N = a.N;

  // shared memory: mirrors [2][E] | stage [E + 2(HW + w)] | taps [w + 1] | obs-step map
  T* mir0 = sm;
  T* mir1 = sm + E;
  T* stage = sm + 2 * E;
  const int stage_sz = E + 2 * (HW + w);
  T* cf = stage + stage_sz;
  int* omap = reinterpret_cast<int*>(cf + (w + 1));
  const bool omap_smem = (N + 1) <= kObsMapCap;
  for (int j = g.tid; j <= w; j += g.NT) cf[j] = a.bcoef[j];
  if (omap_smem)
    for (int j = g.tid; j <= N; j += g.NT) omap[j] = a.obs_of_t[j];
  auto obs_at = [&](int t) { return omap_smem ? omap[t] : a.obs_of_t[t]; };

  const int p0 = wid * LW - HW + lane * C;  // E position of this lane's first value
  int gi[C];
  {
    int g0 = (g.gbase + p0) % g.n;
    if (g0 < 0) g0 += g.n;
#pragma unroll
    for (int c = 0; c < C; ++c) gi[c] = (g0 + c) % g.n;
  }
  constexpr int kVec = 16 / (int)sizeof(T);
  const bool vec_ok = (g.n % kVec == 0) && (gi[0] % kVec == 0) && (gi[0] + C <= g.n);
  const bool own = lane >= HLN && lane < 32 - HLN;
  const bool in_E = p0 >= 0 && p0 + C <= E;
  const T F = a.F, h = a.dt;
  const T h2 = h * T(0.5), h6 = h / T(6), h3 = h / T(3);
  const bool clus = a.CS > 1;
  const T* trj = a.traj + (long long)member * a.traj_mstride;
  const T* V = a.V ? a.V + voff : nullptr;
  const double* V64 = a.V64 ? a.V64 + voff : nullptr;
  T* stash = a.stash + soff;
  // this warp's observation ranges at step oj: injection (owned positions,
  // two segments) and gather (owned positions inside the CTA tile)
  auto wtab = [&](int oj) { return a.wtab + (((long long)g.rank * nw + wid) * a.nos + oj) * 8; };

  // Refresh after every lane wrote its owned values to mirror m (and a
  // barrier): edge lanes reload from the neighbouring warps; every K steps
  // all positions outside the CTA tile reload from their owners' mirrors.
  auto read_halos = [&](T (&v)[C], T* m, bool cstep) {
    if (cstep) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int p = p0 + c;
        if (p < g.HL || p >= g.HL + g.Town) {
          const int r2 = gi[c] / g.Ttile;
          const int ll = g.HL + gi[c] - r2 * g.Ttile;
          if (!clus || r2 == g.rank) {
            v[c] = m[ll];
          } else {
            const T* rem = cg::this_cluster().map_shared_rank(m, r2);
            v[c] = rem[ll];
          }
        } else if (!own) {
          v[c] = m[p];
        }
      }
    } else if (!own && in_E) {
      run_from_smem_vec<T, C>(m + p0, v);
    }
  };

  // ------------------------------------------- delta_0 = U_B v (v staged with a halo)
  for (int j = g.tid; j < stage_sz; j += g.NT) {
    int gk = (g.gbase - HW - w + j) % g.n;
    if (gk < 0) gk += g.n;
    stage[j] = V64 ? (T)V64[gk] : V[gk];
  }
  __syncthreads();
  T dl[C], xr[C];
  conv_run<T, C>(stage, p0 + HW, w, cf, dl);
  load_run<T, C>(trj, gi, vec_ok, xr);

  auto gather = [&](int oj, const T* m) {
    const int* tb = wtab(oj);
    const int off = g.HL - g.a0;
    for (int k = tb[6] + lane; k < tb[7]; k += 32) stash[k] = a.rinv[k] * m[a.obs_idx[k] + off];
  };
  {
    const int oj = obs_at(0);
    if (oj >= 0) {
      if (own) run_to_smem<T, C>(mir0 + p0, dl);
      __syncwarp();
      gather(oj, mir0);
    }
  }

  // ------------------------------------------------ tangent linear, forward
  // observations per lane loaded a step ahead: with 8 values per lane the
  // registers allow it and it hides the loads; shorter runs keep occupancy
  constexpr int kObsPre = (C >= 8) ? 4 : 0;
  for (int t = 0; t < N; ++t) {
    T pf[C];
    if (t + 1 < N) load_run<T, C>(trj + (long long)(t + 1) * g.n, gi, vec_ok, pf);
    // this warp's gather at t + 1: indices and weights in flight during the step
    const int ojn = obs_at(t + 1);
    int gk0 = 0, gk1 = 0;
    int gidx[kObsPre > 0 ? kObsPre : 1];
    T grin[kObsPre > 0 ? kObsPre : 1];
    if (kObsPre > 0 && ojn >= 0) {
      const int* tb = wtab(ojn);
      gk0 = tb[6];
      gk1 = tb[7];
#pragma unroll
      for (int u = 0; u < kObsPre; ++u) {
        const int k = gk0 + lane + 32 * u;
        gidx[u] = k < gk1 ? __ldg(a.obs_idx + k) : 0;
        grin[u] = k < gk1 ? __ldg(a.rinv + k) : T(0);
      }
    }
    Run<T, C> X, e;
    T Xs[C], es[C], acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = xr[c];
      e.v[c] = dl[c];
    }
    shfl_m2m1p1<T, C>(X);
    shfl_m2m1p1<T, C>(e);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T k = tend(X, c, F);
      const T dk = jvp(X, e, c);
      Xs[c] = xr[c] + h2 * k;
      acc[c] = dk;
      es[c] = dl[c] + h2 * dk;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = Xs[c];
      e.v[c] = es[c];
    }
    shfl_m2m1p1<T, C>(X);
    shfl_m2m1p1<T, C>(e);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T k = tend(X, c, F);
      const T dk = jvp(X, e, c);
      Xs[c] = xr[c] + h2 * k;
      acc[c] += T(2) * dk;
      es[c] = dl[c] + h2 * dk;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = Xs[c];
      e.v[c] = es[c];
    }
    shfl_m2m1p1<T, C>(X);
    shfl_m2m1p1<T, C>(e);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T k = tend(X, c, F);
      const T dk = jvp(X, e, c);
      Xs[c] = xr[c] + h * k;
      acc[c] += T(2) * dk;
      es[c] = dl[c] + h * dk;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X.v[c] = Xs[c];
      e.v[c] = es[c];
    }
    shfl_m2m1p1<T, C>(X);
    shfl_m2m1p1<T, C>(e);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      acc[c] += jvp(X, e, c);
      dl[c] += h6 * acc[c];
    }
    if (t + 1 < N) {
#pragma unroll
      for (int c = 0; c < C; ++c) xr[c] = pf[c];
    }
    // publish, gather, refresh
    const int t1 = t + 1;
    T* m = (t1 & 1) ? mir1 : mir0;
    if (own) run_to_smem<T, C>(m + p0, dl);
    if (ojn >= 0) {
      __syncwarp();
      if constexpr (kObsPre > 0) {
        const int off = g.HL - g.a0;
#pragma unroll
        for (int u = 0; u < kObsPre; ++u) {
          const int k = gk0 + lane + 32 * u;
          if (k < gk1) stash[k] = grin[u] * m[gidx[u] + off];
        }
        for (int k = gk0 + lane + 32 * kObsPre; k < gk1; k += 32) stash[k] = a.rinv[k] * m[a.obs_idx[k] + off];
      } else {
        gather(ojn, m);
      }
    }
    const bool cstep = (t1 % a.K == 0) && (t1 < N);
    sync_cluster_or_block(cstep && clus);
    if (t1 < N) read_halos(dl, m, cstep);
    if (cstep && clus) cg::this_cluster().sync();  // remote reads of m end before it is rewritten
  }
  // every stash entry of the cluster is written before any CTA injects
  sync_cluster_or_block(clus);

  // ------------------------------------------------------ adjoint, backward
  T lam[C];
#pragma unroll
  for (int c = 0; c < C; ++c) lam[c] = T(0);
  // this warp's injection at step t: the two index segments as one list,
  // the first kObsPre per lane loaded ahead (pre_*) by the caller
  int ia0 = 0, na = 0, offa = 0, ib0 = 0, nb = 0, offb = 0;
  int pidx[kObsPre > 0 ? kObsPre : 1];
  T pval[kObsPre > 0 ? kObsPre : 1];
  auto inject_prefetch = [&](int t) {
    if constexpr (kObsPre == 0) return;
    const int oj = obs_at(t);
    na = nb = 0;
    if (oj < 0) return;
    const int* tb = wtab(oj);
    ia0 = tb[0];
    na = tb[1] - tb[0];
    offa = tb[2];
    ib0 = tb[3];
    nb = tb[4] - tb[3];
    offb = tb[5];
#pragma unroll
    for (int u = 0; u < kObsPre; ++u) {
      const int f = lane + 32 * u;
      const int k = f < na ? ia0 + f : ib0 + (f - na);
      const bool ok = f < na + nb;
      pidx[u] = ok ? __ldg(a.obs_idx + k) + (f < na ? offa : offb) : 0;
      pval[u] = ok ? stash[k] : T(0);
    }
  };
  auto inject_refresh = [&](int t) {
    T* m = (t & 1) ? mir1 : mir0;
    if (own) run_to_smem<T, C>(m + p0, lam);
    if constexpr (kObsPre > 0) {
      if (na + nb > 0) {
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kObsPre; ++u)
          if (lane + 32 * u < na + nb) m[pidx[u]] += pval[u];
        for (int f = lane + 32 * kObsPre; f < na + nb; f += 32) {
          const int k = f < na ? ia0 + f : ib0 + (f - na);
          m[a.obs_idx[k] + (f < na ? offa : offb)] += stash[k];
        }
        __syncwarp();
        if (own) run_from_smem_vec<T, C>(m + p0, lam);
      }
    } else {
      const int oj = obs_at(t);
      if (oj >= 0) {
        __syncwarp();
        const int* tb = wtab(oj);
#pragma unroll
        for (int sgm = 0; sgm < 2; ++sgm) {
          const int k1 = tb[3 * sgm + 1], off = tb[3 * sgm + 2];
          for (int k = tb[3 * sgm] + lane; k < k1; k += 32) m[a.obs_idx[k] + off] += stash[k];
        }
        __syncwarp();
        if (own) run_from_smem_vec<T, C>(m + p0, lam);
      }
    }
    const bool cstep = ((N - t) % a.K == 0) && (t > 0);
    sync_cluster_or_block(cstep && clus);
    if (t > 0) read_halos(lam, m, cstep);
    if (cstep && clus) cg::this_cluster().sync();
  };
  inject_prefetch(N);
  inject_refresh(N);
  load_run<T, C>(trj + (long long)(N - 1) * g.n, gi, vec_ok, xr);
  for (int t = N - 1; t >= 0; --t) {
    T pf[C];
    if (t > 0) load_run<T, C>(trj + (long long)(t - 1) * g.n, gi, vec_ok, pf);
    inject_prefetch(t);
    Run<T, C> X1, X2, X3, X4, wv;
    T ln[C], ad[C];
    // stage states of the step from x_t
#pragma unroll
    for (int c = 0; c < C; ++c) X1.v[c] = xr[c];
    shfl_all<T, C>(X1);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      X2.v[c] = xr[c] + h2 * tend(X1, c, F);
      ad[c] = lam[c];  // b4
    }
    shfl_all<T, C>(X2);
#pragma unroll
    for (int c = 0; c < C; ++c) X3.v[c] = xr[c] + h2 * tend(X2, c, F);
    shfl_all<T, C>(X3);
#pragma unroll
    for (int c = 0; c < C; ++c) X4.v[c] = xr[c] + h * tend(X3, c, F);
    shfl_all<T, C>(X4);
    // reverse stage 4: u4 = J4^T b4, b4 = lam (the reverse RK4 step)
#pragma unroll
    for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
    shfl_m1p1p2<T, C>(wv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T u = jtvp(X4, wv, c);
      ln[c] = fma(h6, u, lam[c]);
      ad[c] = fma(h2, u, lam[c]);  // b3
    }
    // reverse stage 3
#pragma unroll
    for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
    shfl_m1p1p2<T, C>(wv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T u = jtvp(X3, wv, c);
      ln[c] = fma(h3, u, ln[c]);
      ad[c] = fma(h2, u, lam[c]);  // b2
    }
    // reverse stage 2
#pragma unroll
    for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
    shfl_m1p1p2<T, C>(wv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T u = jtvp(X2, wv, c);
      ln[c] = fma(h3, u, ln[c]);
      ad[c] = fma(h, u, lam[c]);  // b1
    }
    // reverse stage 1
#pragma unroll
    for (int c = 0; c < C; ++c) wv.v[c] = ad[c];
    shfl_m1p1p2<T, C>(wv);
#pragma unroll
    for (int c = 0; c < C; ++c) lam[c] = fma(h6, jtvp(X1, wv, c), ln[c]);
    if (t > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) xr[c] = pf[c];
    }
    inject_refresh(t);
  }

  // ---------------------------------------------- output U_B lambda_0 (+ v)
  // lambda_0 of every CTA's tile is in its mir0 (t = 0 has parity 0)
  sync_cluster_or_block(clus);
  const bool ident = a.include_identity != 0;
  double* dot = (ident && a.dot_out != nullptr) ? a.dot_out + (long long)col * a.dot_stride : nullptr;
  if (a.OUT64) {
    bhalf_from_mirrors<T, C, double>(a, g, mir0, stage, cf, a.OUT64 + voff, ident ? V64 : nullptr,
                                     ident ? V : nullptr, dot);
  } else {
    bhalf_from_mirrors<T, C, T>(a, g, mir0, stage, cf, a.OUT + voff, ident ? V64 : nullptr, ident ? V : nullptr,
                                dot);
  }
}

template <typename T, int C>
cudaError_t launch_warp(const SweepArgs<T>& a, const SweepPlan& p, cudaStream_t s) {
  auto kern = wsweep_kernel<T, C>;
  static bool attrs_set = false;
  if (!attrs_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
    attrs_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.ncol * p.CS), 1, 1);
  cfg.blockDim = dim3((unsigned)p.A, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (p.CS > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T, int C, bool STG, bool CK = false>
cudaError_t launch_impl(const SweepArgs<T>& a, const SweepPlan& p, cudaStream_t s) {
  auto kern = sweep_kernel<T, C, STG, CK>;
  // function attributes are set once (they are not stream work and must not
  // be issued while a stream is being captured)
  static bool attrs_set = false;
  if (!attrs_set) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
    attrs_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.ncol * p.CS), 1, 1);
  cfg.blockDim = dim3((unsigned)p.A, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (p.CS > 1 && !p.ml) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

size_t sweep_smem_bytes(int A, int C, int w, int elem_bytes) {
  const int E = A * C;
  int stage = kNumEdge * 4 * A;
  if (E + 2 * w + 2 > stage) stage = E + 2 * w + 2;
  const size_t elems = (size_t)E + (size_t)stage + (size_t)(w + 1);
  return elems * (size_t)elem_bytes + (size_t)(kObsMapCap + kObsTabCap) * sizeof(int) + 16;
}

bool plan_sweep_exact(int n, int elem_bytes, int w, int CS, int K, SweepPlan* out, int C) {
  if (C == 0) C = (elem_bytes == 8) ? 4 : 8;
  // instantiated runs: FP64 2 or 4 values per thread, FP32 2, 4 or 8
  if (elem_bytes == 8 ? (C != 2 && C != 4) : (C != 2 && C != 4 && C != 8)) return false;
  out->ml = 0;
  out->warp = 0;
  if (CS < 1 || CS > 16 || K < 1 || K > kMaxRefresh) return false;
  const int Ttile = (n + CS - 1) / CS;
  if ((CS - 1) * Ttile >= n) return false;
  const int HL = 8 * K + 8;
  const int need = Ttile + 2 * HL;
  int A = (need + C - 1) / C;
  A = ((A + 31) / 32) * 32;
  if (A > kMaxThreads) return false;
  const int E = A * C;
  const size_t smem = sweep_smem_bytes(A, C, w, elem_bytes);
  if (smem > 227 * 1024) return false;
  out->CS = CS;
  out->C = C;
  out->A = A;
  out->E = E;
  out->Ttile = Ttile;
  out->HL = HL;
  out->K = K;
  out->smem = smem;
  out->ckpt = 0;
  return true;
}

bool plan_sweep_warp(int n, int elem_bytes, int w, int CS, int K, int C, SweepPlan* out) {
  if (elem_bytes == 8 ? (C != 2 && C != 4) : (C != 4 && C != 8)) return false;
  if (CS < 1 || CS > 16 || K < 1 || K > kMaxRefresh) return false;
  const int LW = 32 * C - 2 * warp_halo(C);
  const int Ttile = (n + CS - 1) / CS;
  if ((CS - 1) * Ttile >= n) return false;
  const int HL = 8 * K + 8;
  const int need = Ttile + 2 * HL;
  const int nw = (need + LW - 1) / LW;
  if (nw * 32 > kWarpMaxThreads) return false;
  const int E = nw * LW;
  if (E > n) return false;  // each warp's range maps to distinct points
  const size_t smem = (size_t)(3 * E + 2 * (warp_halo(C) + w) + w + 1) * (size_t)elem_bytes +
                      (size_t)kObsMapCap * sizeof(int) + 16;
  if (smem > 227 * 1024) return false;
  out->CS = CS;
  out->C = C;
  out->A = nw * 32;
  out->E = E;
  out->Ttile = Ttile;
  out->HL = HL;
  out->K = K;
  out->smem = smem;
  out->ml = 0;
  out->warp = 1;
  out->ckpt = 0;
  return true;
}

void warp_obs_table(const SweepPlan& p, int n, int nos, const int* obs_ptr, const int* obs_idx, int* tab) {
  const int LW = 32 * p.C - 2 * warp_halo(p.C);
  const int nw = p.A / 32;
  auto lower = [&](int j, int g) {
    int lo = obs_ptr[j], hi = obs_ptr[j + 1];
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (obs_idx[mid] < g)
        lo = mid + 1;
      else
        hi = mid;
    }
    return lo;
  };
  for (int r = 0; r < p.CS; ++r) {
    const int a0 = r * p.Ttile;
    const int town = (p.Ttile < n - a0) ? p.Ttile : n - a0;
    const int gbase = ((a0 - p.HL) % n + n) % n;
    for (int wi = 0; wi < nw; ++wi) {
      const int e0 = wi * LW, e1 = e0 + LW;
      const int g0 = gbase + e0, g1 = gbase + e1;  // g1 - g0 = LW <= n
      // gather: owned positions inside the CTA tile [HL, HL + town)
      const int ie0 = e0 > p.HL ? e0 : p.HL;
      const int ie1 = e1 < p.HL + town ? e1 : p.HL + town;
      for (int j = 0; j < nos; ++j) {
        int* t = tab + (((long long)r * nw + wi) * nos + j) * 8;
        t[3] = t[4] = 0;
        t[5] = 0;
        if (g1 <= n) {
          t[0] = lower(j, g0);
          t[1] = lower(j, g1);
          t[2] = -gbase;
        } else if (g0 >= n) {
          t[0] = lower(j, g0 - n);
          t[1] = lower(j, g1 - n);
          t[2] = n - gbase;
        } else {
          t[0] = lower(j, g0);
          t[1] = obs_ptr[j + 1];
          t[2] = -gbase;
          t[3] = obs_ptr[j];
          t[4] = lower(j, g1 - n);
          t[5] = n - gbase;
        }
        if (ie0 < ie1) {
          t[6] = lower(j, a0 + ie0 - p.HL);
          t[7] = lower(j, a0 + ie1 - p.HL);
        } else {
          t[6] = t[7] = 0;
        }
      }
    }
  }
}

bool plan_sweep_ml(int n, int elem_bytes, int w, int K, int A, SweepPlan* out, bool ckpt) {
  const int C = (elem_bytes == 8) ? 4 : 8;
  // default threads: 512 (FP64) or 256 (FP32); checkpointed plans 256, whose
  // shared memory also holds K recomputed states of the region
  if (A <= 0) A = (elem_bytes == 8 && !ckpt) ? 512 : 256;
  if (A % 32 != 0 || A > kMaxThreads || K < 1 || K > kMaxRefresh) return false;
  const int E = A * C;
  const int HL = ckpt ? ckpt_halo(K) : 8 * K + 8;
  const int Ttile = E - 2 * HL;
  if (K < 1 || Ttile < 64) return false;
  size_t smem = sweep_smem_bytes(A, C, w, elem_bytes);
  // a checkpointed plan keeps the K recomputed states of its region
  if (ckpt) smem = ((smem + 15) / 16) * 16 + (size_t)K * E * elem_bytes;
  if (smem > 227 * 1024) return false;
  out->ckpt = ckpt ? K : 0;
  out->CS = (n + Ttile - 1) / Ttile;
  out->C = C;
  out->A = A;
  out->E = E;
  out->Ttile = Ttile;
  out->HL = HL;
  out->K = K;
  out->smem = smem;
  out->ml = 1;
  out->warp = 0;
  return true;
}

bool plan_sweep(int n, int elem_bytes, int w, int min_cs, int K_hint, SweepPlan* out, int C) {
  for (int CS = (min_cs > 1 ? min_cs : 1); CS <= 16; ++CS) {
    const int K = K_hint > 0 ? K_hint : (CS == 1 ? 4 : 8);
    if (plan_sweep_exact(n, elem_bytes, w, CS, K, out, C)) {
      out->ml = 0;
      return true;
    }
  }
  return plan_sweep_ml(n, elem_bytes, w, K_hint > 0 ? K_hint : 16, 0, out);
}

void obs_table(const SweepPlan& p, int n, int nos, const int* obs_ptr, const int* obs_idx, int* tab,
               bool* usable) {
  *usable = p.E <= n;
  if (!*usable) return;
  auto lower = [&](int j, int g) {
    int lo = obs_ptr[j], hi = obs_ptr[j + 1];
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (obs_idx[mid] < g)
        lo = mid + 1;
      else
        hi = mid;
    }
    return lo;
  };
  for (int r = 0; r < p.CS; ++r) {
    const int a0 = r * p.Ttile;
    const int town = (p.Ttile < n - a0) ? p.Ttile : n - a0;
    const int gbase = ((a0 - p.HL) % n + n) % n;
    for (int j = 0; j < nos; ++j) {
      int* t = tab + ((long long)r * nos + j) * 8;
      t[0] = lower(j, a0);
      t[1] = lower(j, a0 + town);
      if (gbase + p.E <= n) {
        t[2] = lower(j, gbase);
        t[3] = lower(j, gbase + p.E);
        t[4] = gbase;
        t[5] = t[6] = 0;
        t[7] = 0;
      } else {
        t[2] = lower(j, gbase);
        t[3] = obs_ptr[j + 1];
        t[4] = gbase;
        t[5] = obs_ptr[j];
        t[6] = lower(j, gbase + p.E - n);
        t[7] = gbase - n;
      }
    }
  }
}

template <typename T>
cudaError_t launch_one(const SweepArgs<T>& a, const SweepPlan& p, cudaStream_t s) {
  // checkpointed launches (multi-launch plans: C = 4 FP64, 8 FP32); the
  // nonlinear sweep only stores the checkpoint rows, which the general
  // kernel does
  if (a.ckpt > 0 && a.mode != MODE_NL) {
    if constexpr (sizeof(T) == 8) {
      if (p.C == 4) return launch_impl<T, 4, false, true>(a, p, s);
    } else {
      if (p.C == 8) return launch_impl<T, 8, false, true>(a, p, s);
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 8) {
    const bool stg = a.stages != nullptr && a.mode != MODE_NL;
    if (p.C == 4) return stg ? launch_impl<T, 4, true>(a, p, s) : launch_impl<T, 4, false>(a, p, s);
    if (p.C == 2) return stg ? launch_impl<T, 2, true>(a, p, s) : launch_impl<T, 2, false>(a, p, s);
  } else {
    if (p.C == 8) return launch_impl<T, 8, false>(a, p, s);
    if (p.C == 4) return launch_impl<T, 4, false>(a, p, s);
    if (p.C == 2) return launch_impl<T, 2, false>(a, p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a0, const SweepPlan& p, cudaStream_t s, T* ml_buf0, T* ml_buf1) {
  SweepArgs<T> a = a0;
  a.CS = p.CS;
  a.Ttile = p.Ttile;
  a.HL = p.HL;
  a.E = p.E;
  a.K = p.K;
  a.ckpt = p.ml ? p.ckpt : 0;
  a.xseg_off = a.ckpt ? (int)(((sweep_smem_bytes(p.A, p.C, a0.w, (int)sizeof(T)) + 15) / 16) * 16) : 0;
  if (a.ncol <= 0) return cudaSuccess;
  if (a.ckpt && a.stages != nullptr && a.mode != MODE_NL) return cudaErrorInvalidValue;
  if (p.warp) {
    if (a.mode != MODE_HVP || a.items != nullptr || a.wtab == nullptr) return cudaErrorInvalidValue;
    a.ml = 0;
    if constexpr (sizeof(T) == 8) {
      if (p.C == 4) return launch_warp<T, 4>(a, p, s);
      if (p.C == 2) return launch_warp<T, 2>(a, p, s);
    } else {
      if (p.C == 8) return launch_warp<T, 8>(a, p, s);
      if (p.C == 4) return launch_warp<T, 4>(a, p, s);
    }
    return cudaErrorInvalidValue;
  }
  if (!p.ml) {
    a.ml = 0;
    return launch_one<T>(a, p, s);
  }
  // multi-launch: chunks of K steps, the state of every column through two
  // global buffers (the launch boundary replaces the halo exchange)
  if (a.items != nullptr || ml_buf0 == nullptr || ml_buf1 == nullptr) return cudaErrorInvalidValue;
  // the closing U_B kernel indexes vectors as contiguous [col][n] rows
  if (a.mode != MODE_NL && (a.out_stride != a.n || (a.mode == MODE_HVP && a.v_stride != a.n)))
    return cudaErrorInvalidValue;
  a.ml = 1;
  a.K = 1 << 30;  // no in-launch refresh
  const int N = a.N, K = p.K;
  T* buf[2] = {ml_buf0, ml_buf1};
  int cur = 0;
  if (a.mode == MODE_NL) {
    for (int t0 = 0; t0 < N; t0 += K) {
      a.f0 = t0;
      a.f1 = (t0 + K < N) ? t0 + K : N;
      a.b0 = a.b1 = 0;
      a.st_in = buf[cur];
      a.st_out = buf[1 - cur];
      cudaError_t e = launch_one<T>(a, p, s);
      if (e != cudaSuccess) return e;
      cur = 1 - cur;
    }
    return cudaSuccess;
  }
  if (a.mode == MODE_HVP) {
    for (int t0 = 0; t0 < N; t0 += K) {
      a.f0 = t0;
      a.f1 = (t0 + K < N) ? t0 + K : N;
      a.b0 = a.b1 = 0;
      a.st_in = buf[cur];
      a.st_out = buf[1 - cur];
      cudaError_t e = launch_one<T>(a, p, s);
      if (e != cudaSuccess) return e;
      cur = 1 - cur;
    }
  }
  // backward in chunks of K steps (checkpointed: aligned on the checkpoints,
  // the last chunk first, possibly shorter)
  for (int t1 = N; t1 > 0; t1 = a.b0) {
    a.f0 = a.f1 = 0;
    a.b1 = t1;
    a.b0 = a.ckpt ? ((t1 - 1) / K) * K : ((t1 - K > 0) ? t1 - K : 0);
    a.st_in = buf[cur];
    a.st_out = buf[1 - cur];
    cudaError_t e = launch_one<T>(a, p, s);
    if (e != cudaSuccess) return e;
    cur = 1 - cur;
  }
  // U_B lambda_0 (+ v)
  const long long total = (long long)a.ncol * a.n;
  long long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  const int ident = (a.mode == MODE_HVP && a.include_identity) ? 1 : 0;
  count_launch();
  if (a.OUT64)
    bhalf_out_kernel<T, double><<<(unsigned)blocks, 256, 0, s>>>(a.n, a.w, a.bcoef, a.ncol, buf[cur], a.V64, a.V,
                                                                  a.OUT64, ident);
  else
    bhalf_out_kernel<T, T><<<(unsigned)blocks, 256, 0, s>>>(a.n, a.w, a.bcoef, a.ncol, buf[cur], a.V64, a.V, a.OUT,
                                                            ident);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !(ident && a.dot_out != nullptr)) return e;
  // v . (H v) per column (the cluster epilogue accumulates it in place);
  // column c of a multi-launch sweep is accumulator c
  const double* vin = a.V64;
  const double* vout = a.OUT64;
  if constexpr (sizeof(T) == 8) {
    if (vin == nullptr) vin = a.V;
    if (vout == nullptr) vout = a.OUT;
  }
  if (vin == nullptr || vout == nullptr || a.dot_stride != kPcgAccStride) return cudaErrorInvalidValue;
  return pcg2_col_dot(a.n, a.ncol, vin, vout, a.col_active, reinterpret_cast<PcgAcc*>(a.dot_out), s);
}

template <typename T>
cudaError_t launch_pcg_persist(const PersistArgs<T>& a0, const SweepPlan& p, cudaStream_t s, int* query) {
  if (a0.M <= 0 || (a0.items != nullptr && a0.nitems <= 0)) return cudaSuccess;
  if (p.ml || p.warp || p.ckpt) return cudaErrorInvalidValue;
  PersistArgs<T> a = a0;
  a.sw.CS = p.CS;
  a.sw.Ttile = p.Ttile;
  a.sw.HL = p.HL;
  a.sw.E = p.E;
  a.sw.K = p.K;
  a.sw.ml = 0;
  a.sw.ckpt = 0;
  a.sw.mode = MODE_HVP;
  a.sw.ncol = a.items != nullptr ? a.nitems : a.M;
  a.sw.col_active = nullptr;
  a.sw.include_identity = 1;
  // the between-sweep scratch (reduction slots, c o w, the r tile) fits the
  // sweep's own shared memory (group mode: the caller checks its largest tile)
  const size_t scratch = 32 * sizeof(double) + (size_t)(((a.kmax + 3) & ~3) + p.Ttile) * sizeof(T);
  if (a.items == nullptr && scratch > p.smem) return cudaErrorInvalidValue;
  if (a.items != nullptr) {  // group buckets: FP64 runs of 4, FP32 runs of 8, no stage store
    if (a.sw.stages != nullptr) return cudaErrorInvalidValue;
    if constexpr (sizeof(T) == 8) {
      if (p.C == 4) return launch_persist_impl<T, 4, false, true>(a, p, s, query);
    } else {
      if (p.C == 8) return launch_persist_impl<T, 8, false, true>(a, p, s, query);
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 8) {
    const bool stg = a.sw.stages != nullptr;
    if (p.C == 4) return stg ? launch_persist_impl<T, 4, true>(a, p, s, query) : launch_persist_impl<T, 4, false>(a, p, s, query);
    if (p.C == 2) return stg ? launch_persist_impl<T, 2, true>(a, p, s, query) : launch_persist_impl<T, 2, false>(a, p, s, query);
  } else {
    if (p.C == 8) return launch_persist_impl<T, 8, false>(a, p, s, query);
    if (p.C == 4) return launch_persist_impl<T, 4, false>(a, p, s, query);
    if (p.C == 2) return launch_persist_impl<T, 2, false>(a, p, s, query);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_pcg_persist<double>(const PersistArgs<double>&, const SweepPlan&, cudaStream_t, int*);
template cudaError_t launch_pcg_persist<float>(const PersistArgs<float>&, const SweepPlan&, cudaStream_t, int*);
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, const SweepPlan&, cudaStream_t, double*, double*);
template cudaError_t launch_sweep<float>(const SweepArgs<float>&, const SweepPlan&, cudaStream_t, float*, float*);

}  // namespace eda
