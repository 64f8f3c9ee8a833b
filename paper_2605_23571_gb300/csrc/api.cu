// C ABI of libeda.so: the EDA handle and the orchestration of the sweeps,
// the Nystrom/LMP build and the batched PCG on one CUDA stream.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "lmp.h"

namespace eda {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace eda

using eda::env_int;
using eda::fail;
using eda::grid_for;
using eda::is_device_ptr;
using eda::read_flag;
using eda::set_plan;

namespace eda {

thread_local std::string g_err;

int fail(eda_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

bool is_device_ptr(const void* ptr) {
  if (ptr == nullptr) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

unsigned grid_for(long long count) {
  long long g = (count + 255) / 256;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (unsigned)g;
}

// Installs a sweep tiling and its observation table.
int set_plan(eda_handle* h, bool fp64, const SweepPlan& pl) {
  std::vector<int> tab((size_t)pl.CS * h->nos * 8);
  bool ok = false;
  eda::obs_table(pl, h->n, h->nos, h->h_obs_ptr.data(), h->h_obs_idx.data(), tab.data(), &ok);
  int*& dt = fp64 ? h->tab64 : h->tab32;
  if (dt) {
    CU(h, cudaStreamSynchronize(h->st));
    CU(h, cudaFree(dt));
    dt = nullptr;
  }
  if (ok) {
    CU(h, cudaMalloc((void**)&dt, tab.size() * sizeof(int)));
    CU(h, cudaMemcpy(dt, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  if (fp64) {
    h->plan64 = pl;
    h->tab64_ok = ok;
  } else {
    h->plan32 = pl;
    h->tab32_ok = ok;
  }
  return EDA_OK;
}

int set_warp_plan(eda_handle* h, bool fp64, const SweepPlan* pl) {
  int*& dt = fp64 ? h->wtab64 : h->wtab32;
  SweepPlan& wp = fp64 ? h->wplan64 : h->wplan32;
  if (dt) {
    CU(h, cudaStreamSynchronize(h->st));
    CU(h, cudaFree(dt));
    dt = nullptr;
  }
  wp = SweepPlan{};
  if (pl == nullptr) return EDA_OK;
  std::vector<int> tab((size_t)pl->CS * (pl->A / 32) * h->nos * 8);
  eda::warp_obs_table(*pl, h->n, h->nos, h->h_obs_ptr.data(), h->h_obs_idx.data(), tab.data());
  CU(h, cudaMalloc((void**)&dt, std::max<size_t>(tab.size(), 1) * sizeof(int)));
  CU(h, cudaMemcpy(dt, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
  wp = *pl;
  return EDA_OK;
}

const SweepPlan& hvp_plan(const eda_handle* h, bool fp64, const int** obs_tab, const int** wtab) {
  const SweepPlan& wp = fp64 ? h->wplan64 : h->wplan32;
  if (wp.warp) {
    *obs_tab = nullptr;
    *wtab = fp64 ? h->wtab64 : h->wtab32;
    return wp;
  }
  *wtab = nullptr;
  *obs_tab = fp64 ? (h->tab64_ok ? h->tab64 : nullptr) : (h->tab32_ok ? h->tab32 : nullptr);
  return fp64 ? h->plan64 : h->plan32;
}

int ensure_ml(eda_handle* h, int ncol, bool fp64) {
  const SweepPlan& pl = fp64 ? h->plan64 : h->plan32;
  if (!pl.ml) return EDA_OK;
  const long long need = (long long)ncol * h->n;
  if (fp64 && need > h->ml64_cap) {
    h->ml64_cap = 0;
    for (int i = 0; i < 2; ++i) {
      if (h->ml64[i]) cudaFree(h->ml64[i]);
      h->ml64[i] = nullptr;
      CU(h, cudaMalloc((void**)&h->ml64[i], need * sizeof(double)));
    }
    h->ml64_cap = need;
  }
  if (!fp64 && need > h->ml32_cap) {
    h->ml32_cap = 0;
    for (int i = 0; i < 2; ++i) {
      if (h->ml32[i]) cudaFree(h->ml32[i]);
      h->ml32[i] = nullptr;
      CU(h, cudaMalloc((void**)&h->ml32[i], need * sizeof(float)));
    }
    h->ml32_cap = need;
  }
  return EDA_OK;
}

int read_flag(eda_handle* h, const int* dflag, int* out) {
  CU(h, cudaMemcpyAsync(h->hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CU(h, cudaStreamSynchronize(h->st));
  *out = *h->hflag;
  return EDA_OK;
}

int env_int(const char* name, int dflt) {
  const char* s = std::getenv(name);
  return (s && *s) ? std::atoi(s) : dflt;
}

}  // namespace eda

namespace {



template <typename T>
cudaError_t dalloc(eda_handle* h, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) h->allocs.push_back((void*)*p);
  return e;
}

// An input array given as host or device memory, seen as device memory.
struct In {
  const void* dev = nullptr;
  void* tmp = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t init(const void* p, size_t bytes, cudaStream_t s) {
    st = s;
    if (p == nullptr || is_device_ptr(p)) {
      dev = p;
      return cudaSuccess;
    }
    cudaError_t e = cudaMallocAsync(&tmp, bytes ? bytes : 1, s);
    if (e != cudaSuccess) return e;
    dev = tmp;
    return cudaMemcpyAsync(tmp, p, bytes, cudaMemcpyHostToDevice, s);
  }
  ~In() {
    if (tmp) cudaFreeAsync(tmp, st);
  }
};

// An output array given as host or device memory.
struct Out {
  void* host = nullptr;
  void* dev = nullptr;
  void* tmp = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  cudaError_t init(void* p, size_t nbytes, cudaStream_t s) {
    st = s;
    bytes = nbytes;
    if (p == nullptr || is_device_ptr(p)) {
      dev = p;
      return cudaSuccess;
    }
    host = p;
    cudaError_t e = cudaMallocAsync(&tmp, nbytes ? nbytes : 1, s);
    dev = tmp;
    return e;
  }
  cudaError_t finish() {
    if (!host) return cudaSuccess;
    return cudaMemcpyAsync(host, tmp, bytes, cudaMemcpyDeviceToHost, st);
  }
  ~Out() {
    if (tmp) cudaFreeAsync(tmp, st);
  }
};

// ----------------------------------------------------------------- small kernels
__global__ void count_nonfinite_kernel(long long count, const double* v, int* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) atomicAdd(flag, 1);
}

__global__ void gamma_kernel(int n, int ell, const double* b, double* Phi) {
  const long long total = (long long)ell * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % n);
    const long long c = i / n;
    Phi[i] = b[(c + 1) * n + g] - b[g];
  }
}

__global__ void axpy_kernel(long long count, double alpha, const double* xv, double* yv) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    yv[i] += alpha * xv[i];
}

template <typename T>
__global__ void sub_kernel(long long count, const double* a, const T* bq, T* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)(a[i] - (double)bq[i]);
}

__global__ void bhalf_apply_kernel(int n, int w, const double* coef, int ncol, const double* V, double* out) {
  const long long total = (long long)ncol * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % n);
    const double* v = V + (i / n) * n;
    double acc = coef[0] * v[g];
    for (int dd = 1; dd <= w; ++dd) {
      int gm = g - dd;
      if (gm < 0) gm += n;
      int gq = g + dd;
      if (gq >= n) gq -= n;
      acc += coef[dd] * (v[gm] + v[gq]);
    }
    out[i] = acc;
  }
}

// xb_j = xt + U_B(eta_0 + eta_j) -- the sum is formed first by twin_sum_kernel
__global__ void twin_sum_kernel(int n, int M, const double* eta, double* out) {
  const long long total = (long long)M * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / n;
    const int g = (int)(i % n);
    out[i] = eta[g] + (j > 0 ? eta[i] : 0.0);
  }
}

__global__ void twin_x_kernel(int n, int M, const double* xt, double* xb) {
  const long long total = (long long)M * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    xb[i] += xt[i % n];
}

__global__ void twin_y_kernel(int p, int M, const double* ytrue, const double* rinv, const double* eta,
                              double* y) {
  const long long total = (long long)M * p;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / p;
    const int kk = (int)(i % p);
    const double e = eta[kk] + (j > 0 ? eta[i] : 0.0);
    y[i] = ytrue[kk] + e / sqrt(rinv[kk]);
  }
}

__global__ void iota_kernel(int count, int* v, int value_mode) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    v[i] = value_mode ? i : 0;
}

// Inner threshold of a refinement round of the mixed solve: the round
// reduces its residual by tau, and needs no less than tol when tol is the
// only criterion (with a certified error bound asked for, the bound may
// need a residual below tol, so no floor then).
__device__ __forceinline__ double inner_tol(double tol, double etol, double tau, double rel) {
  return etol > 0.0 ? tau * rel : fmax(tol, tau * rel);
}

// first inner threshold of the mixed solve
__global__ void set_tolm_kernel(int M, PcgScalars* sc, double tol, double etol, double tau) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
    sc[j].tolm = inner_tol(tol, etol, tau, sc[j].relres);
}

__global__ void export_kernel(int M, const PcgScalars* sc, int* iters, double* relres, int* status,
                              double* errb) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    if (iters) iters[j] = sc[j].iters;
    if (relres) relres[j] = sc[j].relres;
    if (status) status[j] = sc[j].status;
    if (errb) errb[j] = sc[j].errb;
  }
}

__global__ void eig_kernel(int k, const double* D, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) out[i] = 1.0 + D[i];
}

// true-residual bookkeeping of the mixed solve
// FP64 true residual r = b - H x of every member; a member whose true
// residual misses tol is reactivated with the next inner threshold
// max(tol, tau * true relres).
// true-residual bookkeeping of the mixed solve (and of the FP64 solve when a
// certified bound is asked for): FP64 true residual r = b - H x of every
// member, its relative norm and the certified error bound
// ||r|| / (||x|| - ||r||) >= ||x - x*|| / ||x*|| (lambda_min(I + A) >= 1,
// Section 2.3).  A member that met its inner threshold but whose true
// residual misses a requested criterion (tol > 0 on ||r||/||b||, etol > 0
// on the bound) is reactivated, with the next inner threshold
// inner_tol(tol, etol, tau, true relres) when tau > 0 (none otherwise).
__global__ void true_res_kernel(int n, const double* b, const double* hx, const double* x, float* r32,
                                double* r64, PcgScalars* sc, int* active, double tol, double etol, int* nactive,
                                int* need, double tau, int maxit) {
  __shared__ double red[32];
  __shared__ double redx[32];
  const int j = blockIdx.x;
  const double* bj = b + (long long)j * n;
  const double* hj = hx + (long long)j * n;
  const double* xj = x + (long long)j * n;
  float* rj = r32 ? r32 + (long long)j * n : nullptr;
  double* rj64 = r64 + (long long)j * n;
  double s = 0.0, sx = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const double rv = bj[g] - hj[g];
    if (rj) rj[g] = (float)rv;
    rj64[g] = rv;
    s += rv * rv;
    sx += xj[g] * xj[g];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    sx += __shfl_down_sync(0xffffffffu, sx, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = s;
    redx[threadIdx.x >> 5] = sx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, tx = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      t += red[i];
      tx += redx[i];
    }
    const double bn = sc[j].bnorm;
    const double rn = sqrt(t), xn = sqrt(tx);
    const double rel = bn > 0.0 ? rn / bn : 0.0;
    const double errb = (bn == 0.0) ? 0.0 : (xn > rn ? rn / (xn - rn) : __longlong_as_double(0x7ff0000000000000ll));
    sc[j].relres = rel;
    sc[j].errb = errb;
    const bool ok = (bn == 0.0) || ((!(tol > 0.0) || rel <= tol) && (!(etol > 0.0) || errb <= etol));
    if (sc[j].status == EDA_CONVERGED && !ok) {
      // the inner solve met its threshold but the FP64 residual misses a
      // criterion: next refinement round, while the member has iterations left
      sc[j].status = EDA_MAXIT;
      if (sc[j].iters < maxit) {
        sc[j].tolm = tau > 0.0 ? inner_tol(tol, etol, tau, rel) : 0.0;
        active[j] = 1;
        atomicAdd(nactive, 1);
        atomicAdd(need, 1);
      }
    }
  }
}

// sc[j].bnorm = ||b_j|| (the split solve's true residual is relative to b)
__global__ void bnorm_kernel(int n, const double* b, PcgScalars* sc) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const double v = b[(long long)j * n + g];
    s += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    sc[j].bnorm = sqrt(t);
  }
}

// J(x0) = -x0^T (b + r0) / 2 into the first entry of each member's cost
// record (the record is NaN elsewhere until the iterations fill it)
__global__ void cost0_kernel(int n, const double* x, const double* b, const double* r, double* jhist,
                             long long jstride) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const long long i = (long long)j * n + g;
    s += x[i] * (b[i] + r[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    jhist[(long long)j * jstride] = -0.5 * t;
  }
}

// ------------------------------------------------------------- sweep helpers
template <typename T>
SweepArgs<T> base_args(eda_handle* h) {
  SweepArgs<T> a{};
  a.n = h->n;
  a.N = h->N;
  a.F = (T)h->F;
  a.dt = (T)h->dt;
  a.obs_of_t = h->obs_of_t;
  a.obs_ptr = h->obs_ptr;
  a.obs_idx = h->obs_idx;
  a.p = h->p;
  a.w = h->w;
  a.nos = h->nos;
  if constexpr (sizeof(T) == 8) {
    a.traj = h->traj;
    a.rinv = h->rinv;
    a.bcoef = h->bcoef;
    a.obs_tab = h->tab64_ok ? h->tab64 : nullptr;
  } else {
    a.traj = h->traj32;
    a.rinv = h->rinv32;
    a.bcoef = h->bcoef32;
    a.obs_tab = h->tab32_ok ? h->tab32 : nullptr;
  }
  a.traj_mstride = (long long)h->trows * h->n;
  a.M = h->M;
  if constexpr (sizeof(T) == 8) a.stages = h->stg;
  a.stage_astride = (long long)h->M * (h->N + 1) * h->n;
  return a;
}

int ensure_stash(eda_handle* h, int ncol) {
  if (ncol <= h->stash_cols) return EDA_OK;
  if (h->stash) cudaFree(h->stash);
  if (h->stash32) cudaFree(h->stash32);
  h->stash = nullptr;
  h->stash32 = nullptr;
  for (auto& p : h->allocs)
    if (p == (void*)h->stash || p == (void*)h->stash32) p = nullptr;
  const size_t cnt = (size_t)ncol * (size_t)(h->p > 0 ? h->p : 1);
  CU(h, cudaMalloc((void**)&h->stash, cnt * sizeof(double)));
  CU(h, cudaMalloc((void**)&h->stash32, cnt * sizeof(float)));
  h->stash_cols = ncol;
  return EDA_OK;
}

__global__ void trace_cols_kernel(unsigned long long* acc, const int* nactive, int ncol) {
  *acc += (unsigned long long)(nactive ? *nactive : ncol);
}

// Adds the completed event pairs of the trace pool to the totals.
int trace_drain(eda_handle* h) {
  if (h->trace_used == 0) return EDA_OK;
  CU(h, cudaEventSynchronize(h->trace_ev[2 * (h->trace_used - 1) + 1]));
  for (int i = 0; i < h->trace_used; ++i) {
    float ms = 0.f;
    CU(h, cudaEventElapsedTime(&ms, h->trace_ev[2 * i], h->trace_ev[2 * i + 1]));
    h->trace_ms[h->trace_kind[i]] += ms;
    h->trace_calls[h->trace_kind[i]] += 1;
  }
  h->trace_used = 0;
  return EDA_OK;
}

// Opens a traced sweep: column count and the first event of a pair.
int trace_begin(eda_handle* h, int kind, const int* active, int ncol) {
  constexpr int kPairs = 1024;
  if (h->trace_ev.empty()) {
    h->trace_ev.resize(2 * kPairs);
    h->trace_kind.resize(kPairs);
    for (auto& e : h->trace_ev) CU(h, cudaEventCreate(&e));
  }
  if (h->trace_used == kPairs) {
    int rc = trace_drain(h);
    if (rc) return rc;
  }
  eda::count_launch();
  trace_cols_kernel<<<1, 1, 0, h->st>>>(h->trace_cols + kind, active ? h->nactive : nullptr, ncol);
  CU(h, cudaGetLastError());
  h->trace_kind[h->trace_used] = kind;
  CU(h, cudaEventRecord(h->trace_ev[2 * h->trace_used], h->st));
  return EDA_OK;
}

int trace_end(eda_handle* h) {
  CU(h, cudaEventRecord(h->trace_ev[2 * h->trace_used + 1], h->st));
  ++h->trace_used;
  return EDA_OK;
}

int hvp_launch(eda_handle* h, const int* dcols, int ncol, const double* V, double* HV, int ident, bool sw64,
               const int* active, double* dot);

// HV = (ident ? V : 0) + A_{m(c)} V for ncol columns, device pointers, FP64 at
// the interface; FP32 sweeps in EDA_MIXED unless force64.  With tracing on,
// the sweep is bracketed by an event pair (active columns counted on the
// device from the active count).  dot (PCG accumulators) != nullptr: the
// sweep also adds v . (H v) of every active column to them.
int hvp_dev(eda_handle* h, const int* dcols, int ncol, const double* V, double* HV, int ident, bool force64,
            const int* active, double* dot = nullptr) {
  if (ncol <= 0) return EDA_OK;
  int rc = ensure_stash(h, ncol);
  if (rc) return rc;
  const bool sw64 = (h->precision == EDA_FP64 || force64);
  const bool traced = h->trace_on && (h->trace_seen++ % h->trace_every) == 0;
  if (traced) {
    rc = trace_begin(h, sw64 ? 0 : 1, active, ncol);
    if (rc) return rc;
  }
  rc = hvp_launch(h, dcols, ncol, V, HV, ident, sw64, active, dot);
  if (rc) return rc;
  return traced ? trace_end(h) : EDA_OK;
}

int hvp_launch(eda_handle* h, const int* dcols, int ncol, const double* V, double* HV, int ident, bool sw64,
               const int* active, double* dot) {
  if (sw64) {
    SweepArgs<double> a = base_args<double>(h);
    a.mode = eda::MODE_HVP;
    a.ncol = ncol;
    a.col_member = dcols;
    a.col_active = active;
    a.V = V;
    a.v_stride = h->n;
    a.OUT = HV;
    a.out_stride = h->n;
    a.stash = h->stash;
    a.stash_stride = h->p;
    a.include_identity = ident;
    a.dot_out = dot;
    a.dot_stride = eda::kPcgAccStride;
    const SweepPlan& pl = eda::hvp_plan(h, true, &a.obs_tab, &a.wtab);
    CU(h, (eda::ensure_ml(h, a.ncol, true) == EDA_OK) ? eda::launch_sweep<double>(a, pl, h->st, h->ml64[0], h->ml64[1]) : cudaErrorMemoryAllocation);
    return EDA_OK;
  }
  // FP32 sweeps reading and writing the FP64 vectors directly
  SweepArgs<float> a = base_args<float>(h);
  a.mode = eda::MODE_HVP;
  a.ncol = ncol;
  a.col_member = dcols;
  a.col_active = active;
  a.V64 = V;
  a.v_stride = h->n;
  a.OUT64 = HV;
  a.out_stride = h->n;
  a.stash = h->stash32;
  a.stash_stride = h->p;
  a.include_identity = ident;
  a.dot_out = dot;
  a.dot_stride = eda::kPcgAccStride;
  const SweepPlan& pl = eda::hvp_plan(h, false, &a.obs_tab, &a.wtab);
  CU(h, (eda::ensure_ml(h, a.ncol, false) == EDA_OK) ? eda::launch_sweep<float>(a, pl, h->st, h->ml32[0], h->ml32[1]) : cudaErrorMemoryAllocation);
  return EDA_OK;
}

// CholeskyQR2 of Y (ell columns): Q (n x ell) and R_Y = R2 R1 (ell x ell).
// Falls back to a shifted first pass when the Gram matrix is not positive
// definite to working precision.
int cholqr2(eda_handle* h, const double* Yin, double* Qout) {
  const int n = h->n, m = h->ell;
  int st = 0;
  CU(h, eda::gemm_tn<double, double>(n, Yin, m, Yin, m, h->G, m, nullptr, true, h->st));
  CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
  CU(h, eda::chol_inv(h->G, m, 0.0, h->R1, h->R1i, h->dstatus, h->st));
  int rc = read_flag(h, h->dstatus, &st);
  if (rc) return rc;
  if (st) {
    // shifted CholeskyQR: G + s I with s proportional to u * ||Y||_F^2
    std::vector<double> Gh((size_t)m * m);
    CU(h, cudaMemcpyAsync(Gh.data(), h->G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(h, cudaStreamSynchronize(h->st));
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr += Gh[(size_t)i * m + i];
    const double shift = 11.0 * ((double)n * m + (double)m * (m + 1)) * 1.1102230246251565e-16 * tr;
    CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
    CU(h, eda::chol_inv(h->G, m, shift, h->R1, h->R1i, h->dstatus, h->st));
    rc = read_flag(h, h->dstatus, &st);
    if (rc) return rc;
    if (st) return fail(h, EDA_ERR_NUMERIC, "sketch QR: Gram matrix not positive definite even after shift");
  }
  CU(h, eda::gemm_nn<double, double>(n, Yin, m, m, h->R1i, nullptr, nullptr, h->Q1, nullptr, h->st));
  CU(h, eda::gemm_tn<double, double>(n, h->Q1, m, h->Q1, m, h->G, m, nullptr, true, h->st));
  CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
  CU(h, eda::chol_inv(h->G, m, 0.0, h->R2, h->R2i, h->dstatus, h->st));
  rc = read_flag(h, h->dstatus, &st);
  if (rc) return rc;
  if (st) return fail(h, EDA_ERR_NUMERIC, "sketch QR: second CholeskyQR pass failed");
  CU(h, eda::gemm_nn<double, double>(n, h->Q1, m, m, h->R2i, nullptr, nullptr, Qout, nullptr, h->st));
  CU(h, eda::tri_mul(h->R2, h->R1, h->RY, m, h->st));
  return EDA_OK;
}

int check_finite(eda_handle* h, const double* v, long long count, const char* what) {
  CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
  eda::count_launch();
  count_nonfinite_kernel<<<grid_for(count), 256, 0, h->st>>>(count, v, h->dstatus);
  CU(h, cudaGetLastError());
  int bad = 0;
  int rc = read_flag(h, h->dstatus, &bad);
  if (rc) return rc;
  if (bad) return fail(h, EDA_ERR_NUMERIC, std::string("non-finite values in ") + what);
  return EDA_OK;
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================

extern "C" {

EDA_API const char* eda_version(void) { return "eda-gb300 0.1 (sm_103a)"; }

EDA_API long long eda_kernel_launches(void) { return eda::g_launches.load(std::memory_order_relaxed); }

EDA_API int eda_trace(eda_handle* h, int enable) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (enable < 0) return fail(h, EDA_ERR_INVALID, "eda_trace: enable < 0");
  if (enable) {
    h->trace_every = enable;
    h->trace_seen = 0;
    int rc = trace_drain(h);
    if (rc) return rc;
    h->trace_ms[0] = h->trace_ms[1] = 0.0;
    h->trace_calls[0] = h->trace_calls[1] = 0;
    CU(h, cudaMemsetAsync(h->trace_cols, 0, 2 * sizeof(unsigned long long), h->st));
  }
  h->trace_on = enable != 0;
  return EDA_OK;
}

EDA_API int eda_trace_read(eda_handle* h, int fp64, long long* sweeps, long long* columns, double* ms) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  int rc = trace_drain(h);
  if (rc) return rc;
  const int kind = fp64 ? 0 : 1;
  unsigned long long cols = 0;
  CU(h, cudaMemcpyAsync(&cols, h->trace_cols + kind, sizeof(cols), cudaMemcpyDeviceToHost, h->st));
  CU(h, cudaStreamSynchronize(h->st));
  if (sweeps) *sweeps = h->trace_calls[kind];
  if (columns) *columns = (long long)cols;
  if (ms) *ms = h->trace_ms[kind];
  return EDA_OK;
}

extern "C++" {
// Drops the convergence-tail tilings of one precision (0 FP64, 1 FP32).
void free_tails(eda_handle* h, int which) {
  for (auto& t : h->tail[which])
    if (t.tab) cudaFree(t.tab);
  h->tail[which].clear();
}

// How many clusters of the persistent PCG on tiling pl fit on the device at
// once (0: it cannot run there).
template <typename TS>
int persist_fits(eda_handle* h, const SweepPlan& pl) {
  eda::PersistArgs<TS> pa{};
  pa.sw = base_args<TS>(h);
  pa.M = h->M;
  pa.kmax = std::max(h->k, 1);
  int q = 0;
  if (eda::launch_pcg_persist<TS>(pa, pl, h->st, &q) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return q;
}

// Tilings for the persistent PCG's convergence tail: at active counts R
// falling by an eighth at a time from 7M/8 to 1 (EDA_TAIL_DIV=d: by R/d from
// M - M/d), times the Hessian-product sweep of R
// active columns on the chosen tiling and on clusters of more CTAs (up to
// 16) with neighbouring refresh periods, and keeps a level's fastest tiling
// where it beats the chosen one by more than 7 %.  The chosen tiling is
// installed again at the end.
int tune_tails(eda_handle* h, bool fp64, cudaEvent_t e0, cudaEvent_t e1) {
  const int which = fp64 ? 0 : 1;
  free_tails(h, which);
  const SweepPlan main = fp64 ? h->plan64 : h->plan32;
  const bool wp = fp64 ? h->wplan64.warp : h->wplan32.warp;
  const int M = h->M;
  if (main.ml || main.warp || main.ckpt || wp || M < 2 || !env_int("EDA_PERSIST", 1) || !env_int("EDA_TAIL", 1))
    return EDA_OK;
  int* mask = nullptr;
  CU(h, cudaMalloc((void**)&mask, (size_t)M * sizeof(int)));
  std::vector<int> hm((size_t)M);
  const int reps = 3;
  int rc = EDA_OK;
  auto time_plan = [&](const SweepPlan& pl, float* ms) -> int {
    int r = set_plan(h, fp64, pl);
    for (int rep = -1; rep < reps && r == EDA_OK; ++rep) {
      if (rep == 0) CU(h, cudaEventRecord(e0, h->st));
      r = hvp_dev(h, h->cols, M, h->pv, h->q, 1, fp64, mask);
    }
    if (r) return r;
    CU(h, cudaEventRecord(e1, h->st));
    CU(h, cudaEventSynchronize(e1));
    CU(h, cudaEventElapsedTime(ms, e0, e1));
    *ms /= reps;
    return EDA_OK;
  };
  const int div = std::max(2, env_int("EDA_TAIL_DIV", 8));  // levels fall by R / div
  for (int R = M - std::max(1, M / div); rc == EDA_OK && R >= 1; R -= std::max(1, R / div)) {
    for (int i = 0; i < M; ++i) hm[(size_t)i] = i < R ? 1 : 0;
    CU(h, cudaMemcpy(mask, hm.data(), (size_t)M * sizeof(int), cudaMemcpyHostToDevice));
    float base_ms = 0.f;
    rc = time_plan(main, &base_ms);
    if (rc) break;
    SweepPlan best = main;
    float best_ms = base_ms;
    for (int CS = main.CS + 1; CS <= 16 && rc == EDA_OK; ++CS)
      for (int K : {main.K / 2, main.K, main.K * 2}) {
        SweepPlan pl;
        if (K < 1 || !eda::plan_sweep_exact(h->n, fp64 ? 8 : 4, h->w, CS, K, &pl, main.C)) continue;
        if (pl.HL > h->n) continue;
        if ((fp64 ? persist_fits<double>(h, pl) : persist_fits<float>(h, pl)) < 1) continue;
        float ms = 0.f;
        rc = time_plan(pl, &ms);
        if (rc) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = pl;
        }
      }
    if (rc) break;
    if (best_ms < 0.93f * base_ms) {
      eda_handle::TailPlan t;
      t.level = R;
      t.plan = best;
      std::vector<int> tab((size_t)best.CS * h->nos * 8);
      bool ok = false;
      eda::obs_table(best, h->n, h->nos, h->h_obs_ptr.data(), h->h_obs_idx.data(), tab.data(), &ok);
      if (ok && !tab.empty()) {
        cudaError_t e = cudaMalloc((void**)&t.tab, tab.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(t.tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
          if (t.tab) cudaFree(t.tab);
          cudaFree(mask);
          return fail(h, EDA_ERR_CUDA, cudaGetErrorString(e));
        }
      }
      h->tail[which].push_back(t);
      if (env_int("EDA_VERBOSE", 0))
        std::fprintf(stderr, "eda_autotune: %s tail at <= %d active: CS=%d K=%d A=%d %.4f ms (chosen tiling %.4f)\n",
                     fp64 ? "FP64" : "FP32", R, best.CS, best.K, best.A, best_ms, base_ms);
    }
  }
  cudaFree(mask);
  int r2 = set_plan(h, fp64, main);
  if (rc) {
    free_tails(h, which);
    return rc;
  }
  return r2;
}
}  // extern "C++"

EDA_API int eda_autotune(eda_handle* h, int which, double* best_ms_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return fail(h, EDA_ERR_STATE, "eda_autotune before eda_set_trajectory");
  if (which == 0) which = (h->precision == EDA_FP64) ? 1 : 3;
  const size_t cnt = (size_t)h->M * h->n;
  cudaEvent_t e0, e1;
  CU(h, cudaEventCreate(&e0));
  CU(h, cudaEventCreate(&e1));
  const int Ks[] = {2, 4, 8, 16};
  double best_total = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fp64 = (pass == 0);
    if (!(which & (fp64 ? 1 : 2))) continue;
    if (!fp64 && h->precision != EDA_MIXED) continue;
    CU(h, cudaMemcpyAsync(h->pv, h->b, cnt * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    const SweepPlan keep = fp64 ? h->plan64 : h->plan32;
    SweepPlan best = keep;
    float best_ms = 1e30f;
    const int reps = fp64 ? 1 : 3;
    // candidates: single-launch cluster plans (CS 1..8, two run lengths),
    // then multi-launch plans where a column spans several tiles
    std::vector<SweepPlan> cands;
    if (h->ckpt > 0) {  // checkpointed: multi-launch plans of K = ckpt_every steps only
      for (int A : {128, 256, 512}) {
        SweepPlan pl;
        if (eda::plan_sweep_ml(h->n, fp64 ? 8 : 4, h->w, h->ckpt, A, &pl, true)) cands.push_back(pl);
      }
    }
    // FP64 sweeps are bound by the FP64 pipe: a refresh every step (K = 1)
    // trades a cluster barrier per step for a narrower halo of redundant work
    std::vector<int> Kc(std::begin(Ks), std::end(Ks));
    if (fp64) Kc.insert(Kc.begin(), 1);
    std::vector<int> Cc = fp64 ? std::vector<int>{4, 2} : std::vector<int>{8, 4, 2};  // values per thread
    for (int C : Cc)
      if (h->ckpt == 0)
      for (int CS = 1; CS <= 8; ++CS)
        for (int K : Kc) {
          SweepPlan pl;
          if (!eda::plan_sweep_exact(h->n, fp64 ? 8 : 4, h->w, CS, K, &pl, C)) continue;
          if (pl.HL > h->n && CS > 1) continue;
          cands.push_back(pl);
        }
    for (int A : {128, 256, 512})
      for (int K : Ks) {
        SweepPlan pl;
        if (h->ckpt == 0 && eda::plan_sweep_ml(h->n, fp64 ? 8 : 4, h->w, 2 * K, A, &pl) && pl.CS >= 2)
          cands.push_back(pl);
      }
    // warp-tiled plans (Hessian-product sweeps only)
    for (int C : {fp64 ? 4 : 8, fp64 ? 2 : 4})
      if (h->ckpt == 0)
      for (int CS = 2; CS <= 16; ++CS)
        for (int K : {4, 8, 16}) {
          SweepPlan pl;
          if (eda::plan_sweep_warp(h->n, fp64 ? 8 : 4, h->w, CS, K, C, &pl)) cands.push_back(pl);
        }
    for (const SweepPlan& pl : cands) {
      int rc = eda::set_warp_plan(h, fp64, pl.warp ? &pl : nullptr);
      if (!rc && !pl.warp) rc = set_plan(h, fp64, pl);
      if (rc) return rc;
      float ms = 0.f;
      for (int rep = -1; rep < reps; ++rep) {
        if (rep == 0) CU(h, cudaEventRecord(e0, h->st));
        rc = hvp_dev(h, h->cols, h->M, h->pv, h->q, 1, fp64, nullptr);
        if (rc) return rc;
      }
      CU(h, cudaEventRecord(e1, h->st));
      CU(h, cudaEventSynchronize(e1));
      CU(h, cudaEventElapsedTime(&ms, e0, e1));
      ms /= reps;
      if (ms < best_ms) {
        best_ms = ms;
        best = pl;
      }
    }
    // the general plan serves the other sweeps; a warp-tiled winner serves
    // the Hessian products beside it
    int rc = set_plan(h, fp64, best.warp ? keep : best);
    if (!rc) rc = eda::set_warp_plan(h, fp64, best.warp ? &best : nullptr);
    if (rc) return rc;
    best_total += best_ms;
    if (env_int("EDA_VERBOSE", 0))
      std::fprintf(stderr, "eda_autotune: %s sweep %s CS=%d K=%d A=%d E=%d C=%d %.4f ms\n", fp64 ? "FP64" : "FP32",
                   best.warp ? "warp-tiled" : (best.ml ? "multi-launch" : "cluster"), best.CS, best.K, best.A, best.E,
                   best.C, best_ms);
    rc = tune_tails(h, fp64, e0, e1);
    if (rc) return rc;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_ms_out) *best_ms_out = best_total;
  return EDA_OK;
}

EDA_API int eda_time_hvp_sweep(eda_handle* h, int reps, int fp64, double* ms_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return fail(h, EDA_ERR_STATE, "eda_time_hvp_sweep before eda_set_trajectory");
  if (reps < 1 || !ms_out) return fail(h, EDA_ERR_INVALID, "eda_time_hvp_sweep: invalid argument");
  const bool use64 = fp64 || h->precision == EDA_FP64;
  const size_t cnt = (size_t)h->M * h->n;
  CU(h, cudaMemcpyAsync(h->pv, h->b, cnt * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  cudaEvent_t e0, e1;
  CU(h, cudaEventCreate(&e0));
  CU(h, cudaEventCreate(&e1));
  int rc = EDA_OK;
  float ms = 0.f;
  for (int rep = -1; rep < reps && rc == EDA_OK; ++rep) {
    if (rep == 0) CU(h, cudaEventRecord(e0, h->st));
    rc = hvp_dev(h, h->cols, h->M, h->pv, h->q, 1, use64, nullptr);
  }
  CU(h, cudaEventRecord(e1, h->st));
  CU(h, cudaEventSynchronize(e1));
  CU(h, cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *ms_out = (double)ms / reps;
  return EDA_OK;
}

EDA_API const char* eda_last_error(const eda_handle* h) { return h ? h->err.c_str() : eda::g_err.c_str(); }

EDA_API int eda_bhalf_gaussian(int n, double length_scale, double sigma_b, double* taps_out, int max_taps,
                               int* w_out) {
  if (n < 1 || !(length_scale > 0.0) || !(sigma_b > 0.0) || !taps_out || max_taps < 1 || !w_out)
    return fail(nullptr, EDA_ERR_INVALID, "eda_bhalf_gaussian: invalid argument");
  const double L = length_scale;
  int wcut = (int)std::floor(L * std::sqrt(-std::log(1e-17)));
  int w = (n - 1) / 2;
  if (wcut < w) w = wcut;
  if (w < 0) w = 0;
  if (w + 1 > max_taps) return fail(nullptr, EDA_ERR_INVALID, "eda_bhalf_gaussian: max_taps too small");
  const double c0 = sigma_b * std::pow(2.0 / (M_PI * L * L), 0.25);
  for (int dd = 0; dd <= w; ++dd) taps_out[dd] = c0 * std::exp(-(double)dd * dd / (L * L));
  *w_out = w;
  return EDA_OK;
}

EDA_API int eda_create(const eda_config* cfg, eda_handle** out) {
  if (!out) return fail(nullptr, EDA_ERR_INVALID, "eda_create: out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, EDA_ERR_INVALID, "eda_create: cfg is NULL");
  const eda_config& c = *cfg;
  if (c.n < 4) return fail(nullptr, EDA_ERR_INVALID, "n must be >= 4");
  if (c.nsteps < 1) return fail(nullptr, EDA_ERR_INVALID, "nsteps must be >= 1");
  if (!std::isfinite(c.F) || !(c.dt > 0.0) || !std::isfinite(c.dt))
    return fail(nullptr, EDA_ERR_INVALID, "F and dt must be finite, dt > 0");
  if (c.n_obs_times < 1 || !c.obs_steps || !c.obs_ptr || !c.obs_idx || !c.rinv)
    return fail(nullptr, EDA_ERR_INVALID, "observation network missing");
  if (c.n_members < 1) return fail(nullptr, EDA_ERR_INVALID, "n_members must be >= 1");
  if (c.bhalf_w < 0 || c.bhalf_w > (c.n - 1) / 2 || !c.bhalf_coef)
    return fail(nullptr, EDA_ERR_INVALID, "bhalf_w must be in [0, (n-1)/2] with coefficients");
  if (c.ell < 0 || c.ell > c.n_members - 1 || c.ell > 80 || c.ell > c.n)
    return fail(nullptr, EDA_ERR_INVALID, "ell must be in [0, min(L, 80, n)]");
  if (c.ell > 0 && (c.k < 1 || c.k > c.ell)) return fail(nullptr, EDA_ERR_INVALID, "k must be in [1, ell]");
  if (c.theta_mode < 0 || c.theta_mode > 2) return fail(nullptr, EDA_ERR_INVALID, "bad theta_mode");
  if (c.theta_mode == EDA_THETA_GIVEN && !(c.theta > 0.0)) return fail(nullptr, EDA_ERR_INVALID, "theta must be > 0");
  if (c.precision != EDA_FP64 && c.precision != EDA_MIXED) return fail(nullptr, EDA_ERR_INVALID, "bad precision");
  if (c.ckpt_every < 0 || c.ckpt_every > eda::kMaxRefresh)
    return fail(nullptr, EDA_ERR_INVALID, "ckpt_every must be in [0, 4096]");
  // observation network
  int prev = -1;
  for (int j = 0; j < c.n_obs_times; ++j) {
    if (c.obs_steps[j] <= prev || c.obs_steps[j] < 0 || c.obs_steps[j] > c.nsteps)
      return fail(nullptr, EDA_ERR_INVALID, "obs_steps must be strictly increasing in [0, nsteps]");
    prev = c.obs_steps[j];
  }
  if (c.obs_ptr[0] != 0) return fail(nullptr, EDA_ERR_INVALID, "obs_ptr[0] must be 0");
  for (int j = 0; j < c.n_obs_times; ++j) {
    if (c.obs_ptr[j + 1] < c.obs_ptr[j]) return fail(nullptr, EDA_ERR_INVALID, "obs_ptr must be non-decreasing");
    int last = -1;
    for (int kk = c.obs_ptr[j]; kk < c.obs_ptr[j + 1]; ++kk) {
      if (c.obs_idx[kk] <= last || c.obs_idx[kk] >= c.n)
        return fail(nullptr, EDA_ERR_INVALID, "obs_idx must be strictly increasing in [0, n) per step");
      last = c.obs_idx[kk];
      if (!(c.rinv[kk] > 0.0) || !std::isfinite(c.rinv[kk]))
        return fail(nullptr, EDA_ERR_INVALID, "rinv must be positive and finite");
    }
  }
  const int p = c.obs_ptr[c.n_obs_times];
  if (p < 1) return fail(nullptr, EDA_ERR_INVALID, "no observations");
  for (int dd = 0; dd <= c.bhalf_w; ++dd)
    if (!std::isfinite(c.bhalf_coef[dd])) return fail(nullptr, EDA_ERR_INVALID, "bhalf_coef not finite");

  eda_handle* h = new eda_handle();
  h->n = c.n;
  h->N = c.nsteps;
  h->M = c.n_members;
  h->p = p;
  h->nos = c.n_obs_times;
  h->w = c.bhalf_w;
  h->ell = c.ell;
  h->k = c.ell > 0 ? c.k : 0;
  h->theta_mode = c.theta_mode;
  h->theta_given = c.theta;
  h->precision = c.precision;
  h->ckpt = c.ckpt_every;
  h->F = c.F;
  h->dt = c.dt;
  h->st = (cudaStream_t)c.stream;

  auto bail = [&](int code) {
    eda_destroy(h);
    return code;
  };
#define CUC(...)                                                                                 \
  do {                                                                                           \
    cudaError_t e__ = (__VA_ARGS__);                                                             \
    if (e__ != cudaSuccess) {                                                                    \
      fail(nullptr, EDA_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__));   \
      return bail(EDA_ERR_CUDA);                                                                 \
    }                                                                                            \
  } while (0)

  // Sweep tiling: a single-launch cluster plan where one fits, else the
  // multi-launch plan.  EDA_SWEEP_K fixes the refresh period;
  // EDA_SWEEP_CS64/CS32 the smallest cluster size; EDA_SWEEP_C64/C32 the
  // values per thread; EDA_SWEEP_ML=<threads> forces multi-launch tiles of
  // that many threads.
  const int Kh = env_int("EDA_SWEEP_K", 0);
  const int cs64 = env_int("EDA_SWEEP_CS64", 1), cs32 = env_int("EDA_SWEEP_CS32", 1);
  const int mlA = env_int("EDA_SWEEP_ML", 0);
  const int c64 = env_int("EDA_SWEEP_C64", 0), c32 = env_int("EDA_SWEEP_C32", 0);
  // A checkpointed trajectory runs multi-launch plans of K = ckpt_every steps
  // (each launch recomputes its segment from the checkpoint).
  const bool planned =
      h->ckpt > 0 ? ((eda::plan_sweep_ml(h->n, 8, h->w, h->ckpt, mlA, &h->plan64, true) ||
                      eda::plan_sweep_ml(h->n, 8, h->w, h->ckpt, 128, &h->plan64, true)) &&
                     (eda::plan_sweep_ml(h->n, 4, h->w, h->ckpt, mlA, &h->plan32, true) ||
                      eda::plan_sweep_ml(h->n, 4, h->w, h->ckpt, 128, &h->plan32, true)))
      : mlA > 0   ? (eda::plan_sweep_ml(h->n, 8, h->w, Kh > 0 ? Kh : 16, mlA, &h->plan64) &&
                   eda::plan_sweep_ml(h->n, 4, h->w, Kh > 0 ? Kh : 16, mlA, &h->plan32))
                  : (eda::plan_sweep(h->n, 8, h->w, cs64, Kh, &h->plan64, c64) &&
                     eda::plan_sweep(h->n, 4, h->w, cs32, Kh, &h->plan32, c32));
  if (!planned) {
    fail(nullptr, EDA_ERR_INVALID, "state size too large for the sweep tiling");
    return bail(EDA_ERR_INVALID);
  }
  // EDA_SWEEP_WARP=1: warp-tiled Hessian-product sweeps (cluster size from
  // EDA_SWEEP_CS64/CS32 upwards, refresh period EDA_SWEEP_K or 8, values per
  // lane EDA_SWEEP_C64/C32), where such a tiling fits
  SweepPlan wp64{}, wp32{};
  bool want_w64 = false, want_w32 = false;
  if (env_int("EDA_SWEEP_WARP", 0) && h->ckpt == 0) {
    const int Kw = Kh > 0 ? Kh : 8;
    for (int cs = std::max(cs64, 2); cs <= 16 && !want_w64; ++cs)
      want_w64 = eda::plan_sweep_warp(h->n, 8, h->w, cs, Kw, c64 ? c64 : 4, &wp64);
    for (int cs = std::max(cs32, 2); cs <= 16 && !want_w32; ++cs)
      want_w32 = eda::plan_sweep_warp(h->n, 4, h->w, cs, Kw, c32 ? c32 : 8, &wp32);
  }

  h->h_obs_ptr.assign(c.obs_ptr, c.obs_ptr + h->nos + 1);
  h->h_obs_idx.assign(c.obs_idx, c.obs_idx + p);
  h->h_obs_of_t.assign(h->N + 1, -1);
  for (int j = 0; j < c.n_obs_times; ++j) h->h_obs_of_t[c.obs_steps[j]] = j;
  const int n = h->n, N = h->N, M = h->M, ell = h->ell, kk = h->k;
  const int mcols = std::max(M, std::max(ell, 1));
  CUC(dalloc(h, &h->obs_of_t, N + 1));
  CUC(dalloc(h, &h->obs_ptr, h->nos + 1));
  CUC(dalloc(h, &h->obs_idx, p));
  CUC(dalloc(h, &h->rinv, p));
  CUC(dalloc(h, &h->rinv32, p));
  CUC(dalloc(h, &h->bcoef, h->w + 1));
  CUC(dalloc(h, &h->bcoef32, h->w + 1));
  // trajectory store: states 0..N, or the checkpoints x_0, x_c, x_2c, ...
  h->trows = h->ckpt > 0 ? N / h->ckpt + 1 : N + 1;
  CUC(dalloc(h, &h->traj, (size_t)M * h->trows * n));
  if (h->precision == EDA_MIXED) CUC(dalloc(h, &h->traj32, (size_t)M * h->trows * n));
  // stage-state store for the FP64 sweeps, which are bound by the FP64 pipe
  // and gain from not recomputing the stages (EDA_STAGE_STORE=0: recompute).
  // FP32 sweeps always recompute: streaming three more arrays costs them more
  // than the arithmetic saved.
  if (env_int("EDA_STAGE_STORE", 1) && h->ckpt == 0) CUC(dalloc(h, &h->stg, (size_t)7 * M * (N + 1) * n));
  CUC(dalloc(h, &h->d, (size_t)M * p));
  CUC(dalloc(h, &h->rd, (size_t)M * p));
  CUC(dalloc(h, &h->b, (size_t)M * n));
  const int me = std::max(ell, 1);
  CUC(dalloc(h, &h->Phi, (size_t)me * n));
  CUC(dalloc(h, &h->Y, (size_t)me * n));
  CUC(dalloc(h, &h->Q1, (size_t)me * n));
  CUC(dalloc(h, &h->Q, (size_t)me * n));
  CUC(dalloc(h, &h->G, (size_t)me * me));
  CUC(dalloc(h, &h->R1, (size_t)me * me));
  CUC(dalloc(h, &h->R1i, (size_t)me * me));
  CUC(dalloc(h, &h->R2, (size_t)me * me));
  CUC(dalloc(h, &h->R2i, (size_t)me * me));
  CUC(dalloc(h, &h->RY, (size_t)me * me));
  CUC(dalloc(h, &h->W, (size_t)me * me));
  CUC(dalloc(h, &h->UT, (size_t)me * me));
  CUC(dalloc(h, &h->Dv, me));
  CUC(dalloc(h, &h->cv, me));
  CUC(dalloc(h, &h->theta, 1));
  CUC(dalloc(h, &h->dstatus, 1));
  CUC(dalloc(h, &h->S, (size_t)std::max(kk, 1) * n));
  CUC(dalloc(h, &h->S32, (size_t)std::max(kk, 1) * n));
  CUC(dalloc(h, &h->lmpW, (size_t)std::max(kk, 1) * M));
  CUC(dalloc(h, &h->x, (size_t)M * n));
  CUC(dalloc(h, &h->r, (size_t)M * n));
  CUC(dalloc(h, &h->z, (size_t)M * n));
  CUC(dalloc(h, &h->pv, (size_t)M * n));
  CUC(dalloc(h, &h->q, (size_t)M * n));
  CUC(dalloc(h, &h->sc, M));
  CUC(dalloc(h, &h->active, M));
  CUC(dalloc(h, &h->nactive, 1));
  CUC(dalloc(h, &h->trace_cols, 2));
  CUC(dalloc(h, &h->acc, M));
  CUC(dalloc(h, &h->Wk, (size_t)M * std::max(kk, 1)));
  {
    // the handle's solve is one problem: its row chunks and problem go to
    // the PCG kernels by value (no task tables)
    eda::PcgProb pr{};
    pr.n = n;
    pr.M = M;
    pr.k = kk;
    pr.item0 = 0;
    pr.off0 = 0;
    pr.S = (h->precision == EDA_MIXED) ? (const void*)h->S32 : (const void*)h->S;
    pr.c = h->cv;
    h->pgrid = eda::pcg_single(pr);
  }
  CUC(dalloc(h, &h->cols, mcols));
  CUC(dalloc(h, &h->zeros, mcols));
  CUC(cudaMallocHost((void**)&h->hflag, sizeof(int)));
  CUC(cudaMallocHost((void**)&h->hring, eda_handle::kRing * sizeof(int)));
  for (int i = 0; i < eda_handle::kRing; ++i) CUC(cudaEventCreateWithFlags(&h->ring_ev[i], cudaEventDisableTiming));

  std::vector<float> tmp32(std::max(p, h->w + 1));
  CUC(cudaMemcpyAsync(h->obs_of_t, h->h_obs_of_t.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUC(cudaMemcpyAsync(h->obs_ptr, c.obs_ptr, (h->nos + 1) * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUC(cudaMemcpyAsync(h->obs_idx, c.obs_idx, p * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUC(cudaMemcpyAsync(h->rinv, c.rinv, p * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CUC(cudaMemcpyAsync(h->bcoef, c.bhalf_coef, (h->w + 1) * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CUC(eda::convert<double, float>(p, h->rinv, h->rinv32, h->st));
  CUC(eda::convert<double, float>(h->w + 1, h->bcoef, h->bcoef32, h->st));
  eda::count_launch();
  iota_kernel<<<grid_for(mcols), 256, 0, h->st>>>(mcols, h->cols, 1);
  eda::count_launch();
  iota_kernel<<<grid_for(mcols), 256, 0, h->st>>>(mcols, h->zeros, 0);
  CUC(cudaGetLastError());
  CUC(cudaStreamSynchronize(h->st));
  {
    const SweepPlan p64 = h->plan64, p32 = h->plan32;
    if (set_plan(h, true, p64) != EDA_OK || set_plan(h, false, p32) != EDA_OK ||
        (want_w64 && eda::set_warp_plan(h, true, &wp64) != EDA_OK) ||
        (want_w32 && eda::set_warp_plan(h, false, &wp32) != EDA_OK)) {
      eda::g_err = h->err;
      return bail(EDA_ERR_CUDA);
    }
  }
#undef CUC
  *out = h;
  return EDA_OK;
}

EDA_API int eda_destroy(eda_handle* h) {
  if (!h) return EDA_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  for (void* p : h->allocs)
    if (p) cudaFree(p);
  if (h->stash) cudaFree(h->stash);
  if (h->stash32) cudaFree(h->stash32);
  for (int i = 0; i < 2; ++i) {
    if (h->ml64[i]) cudaFree(h->ml64[i]);
    if (h->ml32[i]) cudaFree(h->ml32[i]);
  }
  if (h->tab64) cudaFree(h->tab64);
  if (h->tab32) cudaFree(h->tab32);
  if (h->wtab64) cudaFree(h->wtab64);
  if (h->wtab32) cudaFree(h->wtab32);
  for (auto& v : h->tail)
    for (auto& t : v)
      if (t.tab) cudaFree(t.tab);
  for (cudaEvent_t e : h->trace_ev)
    if (e) cudaEventDestroy(e);
  if (h->hflag) cudaFreeHost(h->hflag);
  if (h->hring) cudaFreeHost(h->hring);
  for (int i = 0; i < eda_handle::kRing; ++i)
    if (h->ring_ev[i]) cudaEventDestroy(h->ring_ev[i]);
  delete h;
  return EDA_OK;
}

EDA_API int eda_twin(eda_handle* h, const double* x_spin0, int spinup, const double* eta_b,
                     const double* eta_o, double* xb_out, double* y_out, double* xt0_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!x_spin0 || !eta_b || !eta_o || !xb_out || !y_out || spinup < 0)
    return fail(h, EDA_ERR_INVALID, "eda_twin: invalid argument");
  const int n = h->n, M = h->M, p = h->p;
  In xs, eb, eo;
  CU(h, xs.init(x_spin0, (size_t)n * sizeof(double), h->st));
  CU(h, eb.init(eta_b, (size_t)M * n * sizeof(double), h->st));
  CU(h, eo.init(eta_o, (size_t)M * p * sizeof(double), h->st));
  Out oxb, oy, oxt;
  CU(h, oxb.init(xb_out, (size_t)M * n * sizeof(double), h->st));
  CU(h, oy.init(y_out, (size_t)M * p * sizeof(double), h->st));
  CU(h, oxt.init(xt0_out, (size_t)n * sizeof(double), h->st));
  double *xt = nullptr, *ytrue = nullptr, *tmp = nullptr;
  int* nobs = nullptr;
  CU(h, cudaMallocAsync((void**)&xt, (size_t)n * sizeof(double), h->st));
  CU(h, cudaMallocAsync((void**)&ytrue, (size_t)p * sizeof(double), h->st));
  CU(h, cudaMallocAsync((void**)&tmp, (size_t)M * n * sizeof(double), h->st));
  CU(h, cudaMallocAsync((void**)&nobs, (size_t)(spinup + 1) * sizeof(int), h->st));
  // spin-up: no observations
  if (spinup > 0) {
    CU(h, cudaMemsetAsync(nobs, 0xFF, (size_t)(spinup + 1) * sizeof(int), h->st));
    SweepArgs<double> a = base_args<double>(h);
    a.mode = eda::MODE_NL;
    a.N = spinup;
    a.obs_of_t = nobs;
    a.ncol = 1;
    a.x0 = (const double*)xs.dev;
    a.x0_stride = n;
    a.final_out = xt;
    CU(h, (eda::ensure_ml(h, a.ncol, true) == EDA_OK) ? eda::launch_sweep<double>(a, h->plan64, h->st, h->ml64[0], h->ml64[1]) : cudaErrorMemoryAllocation);
  } else {
    CU(h, cudaMemcpyAsync(xt, xs.dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  }
  // truth over the window, observed
  {
    SweepArgs<double> a = base_args<double>(h);
    a.mode = eda::MODE_NL;
    a.ncol = 1;
    a.x0 = xt;
    a.x0_stride = n;
    a.d_out = ytrue;
    CU(h, (eda::ensure_ml(h, a.ncol, true) == EDA_OK) ? eda::launch_sweep<double>(a, h->plan64, h->st, h->ml64[0], h->ml64[1]) : cudaErrorMemoryAllocation);
  }
  eda::count_launch();
  twin_sum_kernel<<<grid_for((long long)M * n), 256, 0, h->st>>>(n, M, (const double*)eb.dev, tmp);
  eda::count_launch();
  bhalf_apply_kernel<<<grid_for((long long)M * n), 256, 0, h->st>>>(n, h->w, h->bcoef, M, tmp, (double*)oxb.dev);
  eda::count_launch();
  twin_x_kernel<<<grid_for((long long)M * n), 256, 0, h->st>>>(n, M, xt, (double*)oxb.dev);
  eda::count_launch();
  twin_y_kernel<<<grid_for((long long)M * p), 256, 0, h->st>>>(p, M, ytrue, h->rinv, (const double*)eo.dev,
                                                               (double*)oy.dev);
  CU(h, cudaGetLastError());
  if (oxt.dev) CU(h, cudaMemcpyAsync(oxt.dev, xt, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(h, cudaFreeAsync(xt, h->st));
  CU(h, cudaFreeAsync(ytrue, h->st));
  CU(h, cudaFreeAsync(tmp, h->st));
  CU(h, cudaFreeAsync(nobs, h->st));
  CU(h, oxb.finish());
  CU(h, oy.finish());
  CU(h, oxt.finish());
  if (oxb.host || oy.host || oxt.host) CU(h, cudaStreamSynchronize(h->st));
  return EDA_OK;
}

EDA_API int eda_set_trajectory(eda_handle* h, const double* xb, const double* y, double* rhs_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!xb || !y) return fail(h, EDA_ERR_INVALID, "eda_set_trajectory: xb and y are required");
  const int n = h->n, M = h->M, p = h->p, N = h->N;
  In ixb, iy;
  CU(h, ixb.init(xb, (size_t)M * n * sizeof(double), h->st));
  CU(h, iy.init(y, (size_t)M * p * sizeof(double), h->st));
  int rc = check_finite(h, (const double*)ixb.dev, (long long)M * n, "xb");
  if (rc) return rc;
  rc = check_finite(h, (const double*)iy.dev, (long long)M * p, "y");
  if (rc) return rc;
  h->have_traj = h->have_sketch = h->have_lmp = false;
  // nonlinear trajectories and innovations (FP64)
  {
    SweepArgs<double> a = base_args<double>(h);
    a.mode = eda::MODE_NL;
    a.ncol = M;
    a.x0 = (const double*)ixb.dev;
    a.x0_stride = n;
    a.traj_out = h->traj;
    a.traj_out_mstride = (long long)h->trows * n;
    a.stage_out = h->stg;
    a.yobs = (const double*)iy.dev;
    a.d_out = h->d;
    a.rd_out = h->rd;
    CU(h, (eda::ensure_ml(h, a.ncol, true) == EDA_OK) ? eda::launch_sweep<double>(a, h->plan64, h->st, h->ml64[0], h->ml64[1]) : cudaErrorMemoryAllocation);
  }
  if (h->precision == EDA_MIXED) {
    CU(h, eda::convert<double, float>((long long)M * h->trows * n, h->traj, h->traj32, h->st));
  }
  // right-hand sides b_j = U_B^T G_j^T R^{-1} d_j (FP64 adjoint sweep)
  {
    SweepArgs<double> a = base_args<double>(h);
    a.mode = eda::MODE_RHS;
    a.ncol = M;
    a.stash = h->rd;
    a.stash_stride = p;
    a.OUT = h->b;
    a.out_stride = n;
    CU(h, (eda::ensure_ml(h, a.ncol, true) == EDA_OK) ? eda::launch_sweep<double>(a, h->plan64, h->st, h->ml64[0], h->ml64[1]) : cudaErrorMemoryAllocation);
  }
  Out orhs;
  CU(h, orhs.init(rhs_out, (size_t)M * n * sizeof(double), h->st));
  if (orhs.dev)
    CU(h, cudaMemcpyAsync(orhs.dev, h->b, (size_t)M * n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(h, orhs.finish());
  if (orhs.host) CU(h, cudaStreamSynchronize(h->st));
  h->have_traj = true;
  return EDA_OK;
}

EDA_API int eda_hvp(eda_handle* h, const int* member_of_col, int ncol, const double* V, double* HV,
                    int include_identity) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return fail(h, EDA_ERR_STATE, "eda_hvp before eda_set_trajectory");
  if (ncol < 0 || (ncol > 0 && (!member_of_col || !V || !HV))) return fail(h, EDA_ERR_INVALID, "eda_hvp: invalid argument");
  if (ncol == 0) return EDA_OK;
  const int n = h->n;
  std::vector<int> hm;
  const int* mptr = member_of_col;
  if (!is_device_ptr(member_of_col)) {
    for (int c = 0; c < ncol; ++c)
      if (member_of_col[c] < 0 || member_of_col[c] >= h->M) return fail(h, EDA_ERR_INVALID, "member_of_col out of range");
  }
  In im, iv;
  CU(h, im.init(mptr, (size_t)ncol * sizeof(int), h->st));
  CU(h, iv.init(V, (size_t)ncol * n * sizeof(double), h->st));
  Out o;
  CU(h, o.init(HV, (size_t)ncol * n * sizeof(double), h->st));
  int rc = hvp_dev(h, (const int*)im.dev, ncol, (const double*)iv.dev, (double*)o.dev, include_identity ? 1 : 0,
                   false, nullptr);
  if (rc) return rc;
  CU(h, o.finish());
  if (o.host) CU(h, cudaStreamSynchronize(h->st));
  return EDA_OK;
}

EDA_API int eda_bhalf_apply(eda_handle* h, int ncol, const double* V, double* OUT) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (ncol < 0 || (ncol > 0 && (!V || !OUT))) return fail(h, EDA_ERR_INVALID, "eda_bhalf_apply: invalid argument");
  if (ncol == 0) return EDA_OK;
  const int n = h->n;
  In iv;
  CU(h, iv.init(V, (size_t)ncol * n * sizeof(double), h->st));
  Out o;
  CU(h, o.init(OUT, (size_t)ncol * n * sizeof(double), h->st));
  eda::count_launch();
  bhalf_apply_kernel<<<grid_for((long long)ncol * n), 256, 0, h->st>>>(n, h->w, h->bcoef, ncol, (const double*)iv.dev,
                                                                     (double*)o.dev);
  CU(h, cudaGetLastError());
  CU(h, o.finish());
  if (o.host) CU(h, cudaStreamSynchronize(h->st));
  return EDA_OK;
}

EDA_API int eda_sketch(eda_handle* h, const double* phi, int q, double* y_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return fail(h, EDA_ERR_STATE, "eda_sketch before eda_set_trajectory");
  if (h->ell < 1) return fail(h, EDA_ERR_INVALID, "eda_sketch: ell = 0");
  if (q < 1) return fail(h, EDA_ERR_INVALID, "eda_sketch: q must be >= 1");
  const int n = h->n, ell = h->ell;
  In iphi;
  CU(h, iphi.init(phi, (size_t)ell * n * sizeof(double), h->st));
  if (phi) {
    CU(h, cudaMemcpyAsync(h->Phi, iphi.dev, (size_t)ell * n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  } else {
    eda::count_launch();
    gamma_kernel<<<grid_for((long long)ell * n), 256, 0, h->st>>>(n, ell, h->b, h->Phi);
    CU(h, cudaGetLastError());
  }
  h->have_sketch = h->have_lmp = false;
  for (int pass = 1; pass <= q; ++pass) {
    int rc = hvp_dev(h, h->zeros, ell, h->Phi, h->Y, 0, false, nullptr);
    if (rc) return rc;
    if (pass < q) {
      rc = cholqr2(h, h->Y, h->Phi);  // Phi = Q_Y (Algorithm 1, power loop)
      if (rc) return rc;
    }
  }
  Out oy;
  CU(h, oy.init(y_out, (size_t)ell * n * sizeof(double), h->st));
  if (oy.dev) CU(h, cudaMemcpyAsync(oy.dev, h->Y, (size_t)ell * n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(h, oy.finish());
  if (oy.host) CU(h, cudaStreamSynchronize(h->st));
  h->have_sketch = true;
  return EDA_OK;
}

EDA_API int eda_build_lmp(eda_handle* h, double* eigvals_out, double* s_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_sketch) return fail(h, EDA_ERR_STATE, "eda_build_lmp before eda_sketch");
  const int n = h->n, m = h->ell, kk = h->k;
  double nu = 0.0;
  // Algorithm 1 with the Cholesky factor of W; on breakdown the Appendix B
  // shift nu = eps ||Y||_F; if that also breaks down (the sketch is
  // numerically rank deficient), the truncated-eigendecomposition variant.
  bool robust = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    int rc = cholqr2(h, h->Y, h->Q);
    if (rc == EDA_ERR_NUMERIC) {
      robust = true;
      break;
    }
    if (rc) return rc;
    CU(h, eda::gemm_tn<double, double>(n, h->Phi, m, h->Y, m, h->W, m, nullptr, false, h->st));
    CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
    CU(h, eda::nystrom_core(h->W, h->RY, m, kk, nu, h->theta_mode, h->theta_given, h->UT, h->Dv, h->cv, h->theta,
                            h->dstatus, h->st));
    int st = 0;
    rc = read_flag(h, h->dstatus, &st);
    if (rc) return rc;
    if (!st) break;
    if (attempt == 1) {
      robust = true;
      break;
    }
    // Appendix B: shift nu = eps ||Y||_F, Y <- Y + nu Phi
    CU(h, eda::gemm_tn<double, double>(n, h->Y, m, h->Y, m, h->G, m, nullptr, true, h->st));
    std::vector<double> Gh((size_t)m * m);
    CU(h, cudaMemcpyAsync(Gh.data(), h->G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(h, cudaStreamSynchronize(h->st));
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr += Gh[(size_t)i * m + i];
    nu = 2.220446049250313e-16 * std::sqrt(tr);
    eda::count_launch();
    axpy_kernel<<<grid_for((long long)m * n), 256, 0, h->st>>>((long long)m * n, nu, h->Phi, h->Y);
    CU(h, cudaGetLastError());
  }
  if (robust) {
    if (nu != 0.0) {  // undo the shift of Y
      eda::count_launch();
      axpy_kernel<<<grid_for((long long)m * n), 256, 0, h->st>>>((long long)m * n, -nu, h->Phi, h->Y);
      CU(h, cudaGetLastError());
      nu = 0.0;
    }
    // W = Phi^T Y; M = U mu^{-1/2} (kept eigenvalues); Z = Y M (into Q);
    // K = Z^T Z; SB = V D^{-1/2}; S' = Z SB (into pv); then one CholeskyQR
    // pass on S' restores orthonormal columns.  Columns k_eff..k-1 of S are
    // zero (c = 0 there: the LMP is the identity on them).
    const double rtol = 1e-12;
    CU(h, eda::gemm_tn<double, double>(n, h->Phi, m, h->Y, m, h->W, m, nullptr, false, h->st));
    CU(h, eda::robust_winv(h->W, m, rtol, h->RY, h->st));
    CU(h, eda::gemm_nn<double, double>(n, h->Y, m, m, h->RY, nullptr, nullptr, h->Q, nullptr, h->st));
    CU(h, eda::gemm_tn<double, double>(n, h->Q, m, h->Q, m, h->G, m, nullptr, true, h->st));
    CU(h, eda::robust_eig(h->G, m, kk, rtol, h->theta_mode, h->theta_given, h->UT, h->Dv, h->cv, h->theta,
                          h->dstatus, h->st));
    int ke = 0;
    int rc = read_flag(h, h->dstatus, &ke);
    if (rc) return rc;
    if (ke < 0 || ke > kk) return fail(h, EDA_ERR_NUMERIC, "Nystrom: truncated-eigendecomposition variant failed");
    if (ke > 0) {
      CU(h, eda::gemm_nn<double, double>(n, h->Q, m, ke, h->UT, nullptr, nullptr, h->pv, nullptr, h->st));
      CU(h, eda::gemm_tn<double, double>(n, h->pv, ke, h->pv, ke, h->G, ke, nullptr, true, h->st));
      CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
      CU(h, eda::chol_inv(h->G, ke, 0.0, h->R1, h->R1i, h->dstatus, h->st));
      int st = 0;
      rc = read_flag(h, h->dstatus, &st);
      if (rc) return rc;
      if (st) return fail(h, EDA_ERR_NUMERIC, "Nystrom: truncated-eigendecomposition variant failed");
      CU(h, eda::gemm_nn<double, double>(n, h->pv, ke, ke, h->R1i, nullptr, nullptr, h->S, nullptr, h->st));
    }
    if (ke < kk) CU(h, cudaMemsetAsync(h->S + (size_t)ke * n, 0, (size_t)(kk - ke) * n * sizeof(double), h->st));
    h->lmp_rank = ke;
    h->nystrom_path = 2;
  } else {
    h->nystrom_path = (nu != 0.0) ? 1 : 0;
    h->lmp_rank = kk;
    // S = Q_Y U_T(:, 1:k)
    CU(h, eda::gemm_nn<double, double>(n, h->Q, m, kk, h->UT, nullptr, nullptr, h->S, nullptr, h->st));
  }
  h->shift_used = nu;
  if (h->precision == EDA_MIXED) CU(h, eda::convert<double, float>((long long)kk * n, h->S, h->S32, h->st));
  Out oe, os;
  CU(h, oe.init(eigvals_out, (size_t)kk * sizeof(double), h->st));
  CU(h, os.init(s_out, (size_t)kk * n * sizeof(double), h->st));
  if (oe.dev) {
    eda::count_launch();
    eig_kernel<<<1, 128, 0, h->st>>>(kk, h->Dv, (double*)oe.dev);
    CU(h, cudaGetLastError());
  }
  if (os.dev) CU(h, cudaMemcpyAsync(os.dev, h->S, (size_t)kk * n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(h, oe.finish());
  CU(h, os.finish());
  if (oe.host || os.host) CU(h, cudaStreamSynchronize(h->st));
  h->have_lmp = true;
  ++h->lmp_version;
  return EDA_OK;
}

EDA_API int eda_set_lmp(eda_handle* h, const double* s_in, const double* eigvals_in) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (h->k < 1) return fail(h, EDA_ERR_INVALID, "eda_set_lmp: the handle has no LMP rank (ell = 0)");
  if (!s_in || !eigvals_in) return fail(h, EDA_ERR_INVALID, "eda_set_lmp: invalid argument");
  const int n = h->n, kk = h->k;
  std::vector<double> ev(kk);
  if (is_device_ptr(eigvals_in)) {
    CU(h, cudaMemcpyAsync(ev.data(), eigvals_in, kk * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(h, cudaStreamSynchronize(h->st));
  } else {
    std::memcpy(ev.data(), eigvals_in, kk * sizeof(double));
  }
  std::vector<double> D(kk), c(kk);
  for (int i = 0; i < kk; ++i) {
    if (!std::isfinite(ev[i]) || ev[i] < 1.0 || (i > 0 && ev[i] > ev[i - 1]))
      return fail(h, EDA_ERR_INVALID, "eda_set_lmp: eigenvalues must be finite, >= 1 and descending");
    D[i] = ev[i] - 1.0;
  }
  const double lamk = ev[kk - 1];
  double th = h->theta_given;
  if (h->theta_mode == EDA_THETA_LAMBDA_K) th = lamk;
  if (h->theta_mode == EDA_THETA_MID) th = 0.5 * (lamk + 1.0);
  for (int i = 0; i < kk; ++i) c[i] = th / (1.0 + D[i]) - 1.0;
  In is;
  CU(h, is.init(s_in, (size_t)kk * n * sizeof(double), h->st));
  CU(h, cudaMemcpyAsync(h->S, is.dev, (size_t)kk * n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(h, cudaMemcpyAsync(h->Dv, D.data(), kk * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CU(h, cudaMemcpyAsync(h->cv, c.data(), kk * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CU(h, cudaMemcpyAsync(h->theta, &th, sizeof(double), cudaMemcpyHostToDevice, h->st));
  if (h->precision == EDA_MIXED) CU(h, eda::convert<double, float>((long long)kk * n, h->S, h->S32, h->st));
  CU(h, cudaStreamSynchronize(h->st));
  h->nystrom_path = 0;
  h->lmp_rank = h->k;
  h->shift_used = 0.0;
  h->have_lmp = true;
  ++h->lmp_version;
  return EDA_OK;
}

}  // extern "C"

namespace {

// One block: *out = a . b over n values (FP64).
__global__ void dot1_kernel(int n, const double* a, const double* b, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out = t;
  }
}

// v = f * r (the next Lanczos vector)
__global__ void lanczos_vec_kernel(int n, const double* r, double f, double* v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = f * r[i];
}

// r -= alpha q
__global__ void lanczos_r_kernel(int n, double alpha, const double* q, double* r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] -= alpha * q[i];
}

// p = r + beta p
__global__ void lanczos_p_kernel(int n, double beta, const double* r, double* p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = r[i] + beta * p[i];
}

// S[c][i] = sum_j Y[j][c] V[j][i] for the k leading Ritz vectors (Y [m x k]
// row-major, V [m][n]).
__global__ void ritz_vec_kernel(int n, int m, int k, const double* Y, const double* V, double* S) {
  const long long total = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / n), i = (int)(e - (long long)c * n);
    double acc = 0.0;
    for (int j = 0; j < m; ++j) acc += Y[(long long)j * k + c] * V[(long long)j * n + i];
    S[e] = acc;
  }
}

// Eigenpairs of a symmetric m x m matrix (row-major, overwritten) by cyclic
// Jacobi rotations: eigenvalues on A's diagonal, eigenvectors in the columns
// of Q.  Each rotation annihilates A[p][q] with tan = sign(z) / (|z| +
// sqrt(z^2 + 1)), z = (A[q][q] - A[p][p]) / (2 A[p][q]).
void jacobi_eigh(int m, std::vector<double>& A, std::vector<double>& Q) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; ++i) {
      diag += A[(size_t)i * m + i] * A[(size_t)i * m + i];
      for (int j = i + 1; j < m; ++j) off += A[(size_t)i * m + j] * A[(size_t)i * m + j];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double z = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (z >= 0.0 ? 1.0 : -1.0) / (std::fabs(z) + std::sqrt(z * z + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < m; ++r) {  // columns p, q
          const double arp = A[(size_t)r * m + p], arq = A[(size_t)r * m + q];
          A[(size_t)r * m + p] = c * arp - sn * arq;
          A[(size_t)r * m + q] = sn * arp + c * arq;
        }
        for (int r = 0; r < m; ++r) {  // rows p, q
          const double apr = A[(size_t)p * m + r], aqr = A[(size_t)q * m + r];
          A[(size_t)p * m + r] = c * apr - sn * aqr;
          A[(size_t)q * m + r] = sn * apr + c * aqr;
        }
        for (int r = 0; r < m; ++r) {
          const double qrp = Q[(size_t)r * m + p], qrq = Q[(size_t)r * m + q];
          Q[(size_t)r * m + p] = c * qrp - sn * qrq;
          Q[(size_t)r * m + q] = sn * qrp + c * qrq;
        }
      }
  }
}

}  // namespace

extern "C" {

EDA_API int eda_ritz_lmp(eda_handle* h, int member, int iters, const double* b, double* ritz_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return fail(h, EDA_ERR_STATE, "eda_ritz_lmp before eda_set_trajectory");
  const int n = h->n, k = h->k;
  if (k < 1) return fail(h, EDA_ERR_INVALID, "eda_ritz_lmp: the handle has no LMP rank (ell = 0)");
  if (member < 0 || member >= h->M || iters < k || iters > 256 || iters > n)
    return fail(h, EDA_ERR_INVALID, "eda_ritz_lmp: member outside [0, L+1) or iters outside [k, min(256, n)]");
  // CG without preconditioner from x0 = 0 on member's Hessian, FP64 sweeps;
  // v_j = (-1)^j r_j / |r_j| and CG's coefficients (Section 3; the
  // CG-Lanczos relation)
  double *V = nullptr, *r = nullptr, *pv = nullptr, *q = nullptr, *d = nullptr, *Yd = nullptr, *Sd = nullptr;
  int* col = nullptr;
  struct Frees {
    std::vector<void*> ps;
    ~Frees() {
      for (void* p : ps)
        if (p) cudaFree(p);
    }
  } frees;
  auto dal = [&](double** p, size_t cnt) -> cudaError_t {
    cudaError_t e = cudaMalloc((void**)p, cnt * sizeof(double));
    if (e == cudaSuccess) frees.ps.push_back(*p);
    return e;
  };
  CU(h, dal(&V, (size_t)iters * n));
  CU(h, dal(&r, n));
  CU(h, dal(&pv, n));
  CU(h, dal(&q, n));
  CU(h, dal(&d, 2));
  CU(h, cudaMalloc((void**)&col, sizeof(int)));
  frees.ps.push_back(col);
  CU(h, cudaMemcpyAsync(col, &member, sizeof(int), cudaMemcpyHostToDevice, h->st));
  In ib;
  CU(h, ib.init(b, (size_t)n * sizeof(double), h->st));
  const double* bm = b ? (const double*)ib.dev : h->b + (long long)member * n;
  CU(h, cudaMemcpyAsync(r, bm, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(h, cudaMemcpyAsync(pv, bm, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  auto dot = [&](const double* a, const double* b2, double* out) -> int {
    eda::count_launch();
    dot1_kernel<<<1, 1024, 0, h->st>>>(n, a, b2, d);
    CU(h, cudaGetLastError());
    double hv = 0.0;
    CU(h, cudaMemcpyAsync(&hv, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(h, cudaStreamSynchronize(h->st));
    *out = hv;
    return EDA_OK;
  };
  double rr = 0.0;
  int rc = dot(r, r, &rr);
  if (rc) return rc;
  if (!(rr > 0.0) || !std::isfinite(rr)) return fail(h, EDA_ERR_NUMERIC, "eda_ritz_lmp: the right-hand side is zero or not finite");
  std::vector<double> alpha((size_t)iters), beta((size_t)iters);
  const unsigned gb = grid_for(n);
  for (int j = 0; j < iters; ++j) {
    eda::count_launch();
    lanczos_vec_kernel<<<gb, 256, 0, h->st>>>(n, r, ((j & 1) ? -1.0 : 1.0) / std::sqrt(rr), V + (long long)j * n);
    CU(h, cudaGetLastError());
    rc = hvp_dev(h, col, 1, pv, q, 1, true, nullptr);
    if (rc) return rc;
    double pq = 0.0;
    rc = dot(pv, q, &pq);
    if (rc) return rc;
    if (!(pq > 0.0) || !std::isfinite(pq)) return fail(h, EDA_ERR_NUMERIC, "eda_ritz_lmp: CG breakdown (p.Hp <= 0)");
    alpha[(size_t)j] = rr / pq;
    eda::count_launch();
    lanczos_r_kernel<<<gb, 256, 0, h->st>>>(n, alpha[(size_t)j], q, r);
    CU(h, cudaGetLastError());
    double rr_new = 0.0;
    rc = dot(r, r, &rr_new);
    if (rc) return rc;
    if (!(rr_new > 0.0) && j + 1 < iters)
      return fail(h, EDA_ERR_NUMERIC, "eda_ritz_lmp: CG converged before the requested iterations");
    beta[(size_t)j] = rr_new / rr;
    eda::count_launch();
    lanczos_p_kernel<<<gb, 256, 0, h->st>>>(n, beta[(size_t)j], r, pv);
    CU(h, cudaGetLastError());
    rr = rr_new;
  }
  // T = V^T H V from CG's coefficients, its eigenpairs on the host
  const int m = iters;
  std::vector<double> T((size_t)m * m, 0.0), Q;
  for (int j = 0; j < m; ++j) {
    T[(size_t)j * m + j] = 1.0 / alpha[(size_t)j] + (j > 0 ? beta[(size_t)j - 1] / alpha[(size_t)j - 1] : 0.0);
    if (j + 1 < m) T[(size_t)j * m + j + 1] = T[(size_t)(j + 1) * m + j] = std::sqrt(beta[(size_t)j]) / alpha[(size_t)j];
  }
  jacobi_eigh(m, T, Q);
  std::vector<int> order((size_t)m);
  for (int i = 0; i < m; ++i) order[(size_t)i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b2) { return T[(size_t)a * m + a] > T[(size_t)b2 * m + b2]; });
  std::vector<double> theta((size_t)m), Y((size_t)m * k);
  for (int i = 0; i < m; ++i) theta[(size_t)i] = T[(size_t)order[(size_t)i] * m + order[(size_t)i]];
  for (int j = 0; j < m; ++j)
    for (int c = 0; c < k; ++c) Y[(size_t)j * k + c] = Q[(size_t)j * m + order[(size_t)c]];
  if (ritz_out) std::memcpy(ritz_out, theta.data(), (size_t)m * sizeof(double));
  // the k leading Ritz vectors S = V Y, installed as the LMP's eigenpairs
  CU(h, dal(&Yd, (size_t)m * k));
  CU(h, dal(&Sd, (size_t)k * n));
  CU(h, cudaMemcpyAsync(Yd, Y.data(), (size_t)m * k * sizeof(double), cudaMemcpyHostToDevice, h->st));
  eda::count_launch();
  ritz_vec_kernel<<<grid_for((long long)k * n), 256, 0, h->st>>>(n, m, k, Yd, V, Sd);
  CU(h, cudaGetLastError());
  std::vector<double> lead(theta.begin(), theta.begin() + k);
  for (double& v : lead)
    if (v < 1.0) v = 1.0;  // Ritz values of I + A lie above 1 up to rounding
  return eda_set_lmp(h, Sd, lead.data());
}

EDA_API int eda_plan_tiling(int n, int fp64, int w, int kind, int cs, int threads, int K, int C, int* info) {
  if (!info || n < 1 || w < 0 || K < 1 || K > eda::kMaxRefresh || kind < 0 || kind > 3)
    return fail(nullptr, EDA_ERR_INVALID, "eda_plan_tiling: invalid argument");
  const int eb = fp64 ? 8 : 4;
  eda::SweepPlan p{};
  bool ok = false;
  if (kind == 0) ok = eda::plan_sweep_exact(n, eb, w, cs, K, &p, C);
  if (kind == 1) ok = C == 0 && eda::plan_sweep_ml(n, eb, w, K, threads, &p);
  if (kind == 2) ok = eda::plan_sweep_warp(n, eb, w, cs, K, C, &p);
  if (kind == 3) ok = C == 0 && eda::plan_sweep_ml(n, eb, w, K, threads, &p, true);
  if (!ok) return fail(nullptr, EDA_ERR_INVALID, "eda_plan_tiling: no tiling of that shape fits");
  info[0] = p.warp ? 2 : (p.ml ? 1 : 0);
  info[1] = p.CS;
  info[2] = p.A;
  info[3] = p.C;
  info[4] = p.K;
  info[5] = p.HL;
  info[6] = p.Ttile;
  info[7] = (int)p.smem;
  return EDA_OK;
}

EDA_API int eda_sweep_plan(eda_handle* h, int fp64, int* info) {
  if (!h || !info) return fail(h, EDA_ERR_INVALID, "handle or info is NULL");
  if (!fp64 && h->precision != EDA_MIXED) return fail(h, EDA_ERR_INVALID, "an FP64 handle has no FP32 sweep");
  const int* ot = nullptr;
  const int* wt = nullptr;
  const eda::SweepPlan& p = eda::hvp_plan(h, fp64 != 0, &ot, &wt);
  info[0] = p.warp ? 2 : (p.ml ? 1 : 0);
  info[1] = p.CS;
  info[2] = p.A;
  info[3] = p.C;
  info[4] = p.K;
  info[5] = p.HL;
  info[6] = p.Ttile;
  info[7] = (int)p.smem;
  return EDA_OK;
}

EDA_API int eda_tail_plans(eda_handle* h, int fp64, int cap, int* count, int* levels, int* info) {
  if (!h || !count || cap < 0) return fail(h, EDA_ERR_INVALID, "eda_tail_plans: invalid argument");
  if (!fp64 && h->precision != EDA_MIXED) return fail(h, EDA_ERR_INVALID, "an FP64 handle has no FP32 sweep");
  const std::vector<eda_handle::TailPlan>& t = h->tail[fp64 ? 0 : 1];
  *count = (int)t.size();
  for (int i = 0; i < (int)t.size() && i < cap; ++i) {
    if (levels) levels[i] = t[(size_t)i].level;
    if (info) {
      const eda::SweepPlan& p = t[(size_t)i].plan;
      int* o = info + 8 * (size_t)i;
      o[0] = 0;
      o[1] = p.CS;
      o[2] = p.A;
      o[3] = p.C;
      o[4] = p.K;
      o[5] = p.HL;
      o[6] = p.Ttile;
      o[7] = (int)p.smem;
    }
  }
  return EDA_OK;
}

EDA_API int eda_set_tail_plan(eda_handle* h, int fp64, int level, int cs, int K, int C) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!fp64 && h->precision != EDA_MIXED) return fail(h, EDA_ERR_INVALID, "an FP64 handle has no FP32 sweep");
  const int which = fp64 ? 0 : 1;
  if (level < 0 || level > h->M) return fail(h, EDA_ERR_INVALID, "eda_set_tail_plan: level outside [0, L+1]");
  if (level == 0) {
    CU(h, cudaStreamSynchronize(h->st));
    free_tails(h, which);
    return EDA_OK;
  }
  const eda::SweepPlan& main = fp64 ? h->plan64 : h->plan32;
  const bool wp = fp64 ? h->wplan64.warp : h->wplan32.warp;
  if (main.ml || main.warp || main.ckpt || wp)
    return fail(h, EDA_ERR_INVALID, "eda_set_tail_plan: the chosen tiling is not a thread-block cluster tiling");
  eda::SweepPlan pl;
  if (!eda::plan_sweep_exact(h->n, fp64 ? 8 : 4, h->w, cs, K, &pl, C == 0 ? main.C : C) || (pl.HL > h->n && cs > 1))
    return fail(h, EDA_ERR_INVALID, "eda_set_tail_plan: no cluster tiling of that shape fits");
  if ((fp64 ? persist_fits<double>(h, pl) : persist_fits<float>(h, pl)) < 1)
    return fail(h, EDA_ERR_INVALID, "eda_set_tail_plan: the persistent PCG cannot run on that tiling");
  eda_handle::TailPlan t;
  t.level = level;
  t.plan = pl;
  std::vector<int> tab((size_t)pl.CS * h->nos * 8);
  bool ok = false;
  eda::obs_table(pl, h->n, h->nos, h->h_obs_ptr.data(), h->h_obs_idx.data(), tab.data(), &ok);
  if (ok && !tab.empty()) {
    CU(h, cudaMalloc((void**)&t.tab, tab.size() * sizeof(int)));
    cudaError_t e = cudaMemcpy(t.tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(t.tab);
      return fail(h, EDA_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  CU(h, cudaStreamSynchronize(h->st));
  std::vector<eda_handle::TailPlan>& v = h->tail[which];
  for (auto it = v.begin(); it != v.end(); ++it)
    if (it->level == level) {
      if (it->tab) cudaFree(it->tab);
      v.erase(it);
      break;
    }
  v.push_back(t);
  std::sort(v.begin(), v.end(), [](const eda_handle::TailPlan& a, const eda_handle::TailPlan& b) {
    return a.level > b.level;
  });
  return EDA_OK;
}

EDA_API int eda_lmp_info(eda_handle* h, int* path, int* rank, double* shift) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_lmp) return fail(h, EDA_ERR_STATE, "eda_lmp_info before eda_build_lmp or eda_set_lmp");
  if (path) *path = h->nystrom_path;
  if (rank) *rank = h->lmp_rank;
  if (shift) *shift = h->shift_used;
  return EDA_OK;
}

}  // extern "C"

namespace {

// How a PCG loop applies the LMP (see pcg_loop_t).
struct LoopMode {
  bool split = false;  // CG on U H U with U = U_theta applied around each product
  bool tc = false;     // the LMP on tensor cores (split-BF16) instead of CUDA cores
};

__global__ void ucoef_kernel(int k, const double* c, double* uv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const double a = sqrt(1.0 + c[i]);  // 1 + c_i = theta / (1 + lambda_i) > 0
    uv[i] = a - 1.0;
    uv[k + i] = 1.0 / a - 1.0;
  }
}

// trace_cols[kind] += sign * (sum of the members' iteration counts): around
// a persistent PCG launch, the member iterations (one swept column each) it ran
__global__ void iters_delta_kernel(unsigned long long* acc, const eda::PcgScalars* sc, int M, int sign) {
  __shared__ long long red[256];
  long long s = 0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) s += sc[m].iters;
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
    *acc += (unsigned long long)(sign * t);
  }
}

// Coefficients of U_theta (sqrt(theta) (1 + lambda_i)^{-1/2} - 1, Section
// 3.1, Eq. (lmp)) and of its inverse, for the current LMP.
int prep_ucoef(eda_handle* h) {
  if (h->uv_version == h->lmp_version) return EDA_OK;
  if (!h->uv) CU(h, dalloc(h, &h->uv, (size_t)2 * std::max(h->k, 1)));
  eda::count_launch();
  ucoef_kernel<<<1, 128, 0, h->st>>>(h->k, h->cv, h->uv);
  CU(h, cudaGetLastError());
  h->uv_version = h->lmp_version;
  return EDA_OK;
}

// BF16 high/low copies of S for the tensor-core LMP, for the current LMP.
int prep_bf16(eda_handle* h) {
  if (h->bf_version == h->lmp_version) return EDA_OK;
  if (!h->Sbf) {
    __nv_bfloat16* p = nullptr;
    CU(h, dalloc(h, &p, eda::lmp_tc_elems(h->n, h->k)));
    h->Sbf = p;
  }
  CU(h, eda::split_bf16(h->n, h->k, h->S, static_cast<__nv_bfloat16*>(h->Sbf), h->st));
  h->bf_version = h->lmp_version;
  return EDA_OK;
}

// Z = R + S diag(coef) S^T R for ncol vectors (device memory, Z may alias
// R; columns with active[c] == 0 untouched when active != nullptr): which 0
// applies P_theta, 1 U_theta, 2 U_theta^{-1}; kind 0 on CUDA cores in the
// handle's LMP precision (FP64, or FP32 in EDA_MIXED), kind 1 split-BF16 on
// tensor cores.
int lmp_apply_dev(eda_handle* h, int which, int kind, int ncol, const double* R, double* Z, const int* active) {
  if (ncol <= 0) return EDA_OK;
  const int n = h->n, k = h->k;
  if (which != 0) {
    int rc = prep_ucoef(h);
    if (rc) return rc;
  }
  const double* coef = which == 0 ? h->cv : (which == 1 ? h->uv : h->uv + k);
  if (kind == 0) {
    const bool f64 = h->precision == EDA_FP64;
    const long long need = (long long)ncol * std::max(k, 1) * (f64 ? 8 : 4);
    if (need > h->wcc_cap) {
      if (h->Wcc) cudaFree(h->Wcc);
      for (auto& p : h->allocs)
        if (p == h->Wcc) p = nullptr;
      h->Wcc = nullptr;
      h->wcc_cap = 0;
      CU(h, cudaMalloc(&h->Wcc, (size_t)need));
      h->wcc_cap = need;
    }
    if (f64)
      CU(h, eda::lmp_apply_cc<double>(n, k, h->S, coef, ncol, R, Z, active, static_cast<double*>(h->Wcc), k, h->st));
    else
      CU(h, eda::lmp_apply_cc<float>(n, k, h->S32, coef, ncol, R, Z, active, static_cast<float*>(h->Wcc), k, h->st));
    return EDA_OK;
  }
  int rc = prep_bf16(h);
  if (rc) return rc;
  const long long need = (long long)((ncol + 15) / 16 * 16) * eda::lmp_tc_kt(k);
  if (need > h->wtc_cap) {
    if (h->Wtc) cudaFree(h->Wtc);
    for (auto& p : h->allocs)
      if (p == (void*)h->Wtc) p = nullptr;
    h->Wtc = nullptr;
    h->wtc_cap = 0;
    CU(h, cudaMalloc((void**)&h->Wtc, (size_t)need * sizeof(float)));
    h->wtc_cap = need;
  }
  if (!h->tc_timeout) {
    CU(h, dalloc(h, &h->tc_timeout, 1));
    CU(h, cudaMemsetAsync(h->tc_timeout, 0, sizeof(int), h->st));
  }
  CU(h, eda::lmp_apply_tc(n, k, static_cast<const __nv_bfloat16*>(h->Sbf), coef, ncol, R, Z, active, h->Wtc,
                          h->tc_timeout, h->st));
  return EDA_OK;
}

// A tensor-core wait that gave up (read after the stream synchronised).
int check_tc_timeout(eda_handle* h) {
  if (!h->tc_timeout) return EDA_OK;
  int t = 0;
  int rc = read_flag(h, h->tc_timeout, &t);
  if (rc) return rc;
  if (t) {
    CU(h, cudaMemsetAsync(h->tc_timeout, 0, sizeof(int), h->st));
    return fail(h, EDA_ERR_TIMEOUT, "tensor-core LMP: a bounded wait for the MMA gave up");
  }
  return EDA_OK;
}

// PCG iterations from the current (x, r) state (the caller has run
// pcg_start): FP64 vectors and scalars; sweeps in FP64 (sweep64) or FP32,
// LMP arithmetic in FP64 or FP32 accordingly.  One iteration is the sweep
// (with p.q in its epilogue) and the update, precond and dir launches over
// row chunks of all members (pcg.h).  The host polls the active count
// through a ring of pinned host slots (the dir launch writes the count) and
// runs at most kRing-1 iterations ahead of the device.
template <typename TS>
int pcg_loop_t(eda_handle* h, double tol, int maxit, int it0, bool use_lmp, int* it_done, bool sweep64,
               int replace_every, const LoopMode& lm) {
  const int M = h->M;
  // no stopping criterion at all (tol = 0, no error bound): exactly maxit iterations
  const int fixed = (tol > 0.0 || h->pgrid.one.etol > 0.0) ? 0 : maxit;
  // the LMP inside the row-chunk kernels (CUDA cores), or z = P r by a
  // separate tensor-core launch pair, or (split) no preconditioner in the
  // kernels and U applied around every product
  const int lmp = (use_lmp && !lm.split && !lm.tc) ? 1 : 0;
  const bool zext = use_lmp && lm.tc && !lm.split;
  const int kind = lm.tc ? 1 : 0;
  const int kmax = std::max(h->k, 1);
  TS* Wk = reinterpret_cast<TS*>(h->Wk);
  // start: z = P r, p = z, r.z
  CU(h, eda::pcg2_reset(h->acc, M, Wk, (size_t)M * kmax * sizeof(TS), h->st));
  CU(h, eda::pcg2_update<TS>(h->pgrid, kmax, M, h->pv, h->q, h->x, h->r, h->sc, h->acc, h->active,
                             Wk, 0, 0, lmp, h->nactive, h->st));
  if (zext) {
    int rc = lmp_apply_dev(h, 0, 1, M, h->r, h->z, h->active);
    if (rc) return rc;
  }
  CU(h, eda::pcg2_precond<TS>(h->pgrid, kmax, M, h->r, h->z, h->pv, h->sc, h->acc, h->active, Wk,
                              0, tol, maxit, fixed, lmp, 1, h->nactive, h->st, zext ? h->z : nullptr));
  // the first update accumulates the projections of r_1 from zero
  CU(h, cudaMemsetAsync(Wk, 0, (size_t)M * kmax * sizeof(TS), h->st));
  // the persistent PCG: the whole loop in one launch (one cluster per
  // member) where the tiling is a cluster plan and nothing per iteration is
  // asked of the host (no cost record, residual replacement or outside LMP)
  const SweepPlan& gp = sweep64 ? h->plan64 : h->plan32;
  const bool wplan = sweep64 ? h->wplan64.warp : h->wplan32.warp;
  if (maxit >= 1 && env_int("EDA_PERSIST", 1) && !lm.split && !lm.tc && replace_every == 0 &&
      h->pgrid.one.jhist == nullptr && !gp.ml && !gp.warp && !gp.ckpt && !wplan) {
    int rc = ensure_stash(h, M);
    if (rc) return rc;
    if (!h->pacc) CU(h, dalloc(h, &h->pacc, (size_t)M));
    if (!h->Wp) {
      double* wp = nullptr;  // 8 bytes per entry serves both precisions
      CU(h, dalloc(h, &wp, (size_t)2 * M * kmax));
      h->Wp = wp;
    }
    CU(h, cudaMemsetAsync(h->pacc, 0, (size_t)M * sizeof(eda::PersistAcc), h->st));
    CU(h, cudaMemsetAsync(h->Wp, 0, (size_t)2 * M * kmax * sizeof(TS), h->st));
    eda::PersistArgs<TS> pa{};
    pa.sw = base_args<TS>(h);
    pa.sw.mode = eda::MODE_HVP;
    pa.sw.ncol = M;
    pa.sw.col_member = h->cols;
    if constexpr (sizeof(TS) == 8) {
      pa.sw.V = h->pv;
      pa.sw.OUT = h->q;
      pa.sw.stash = h->stash;
    } else {
      pa.sw.V64 = h->pv;
      pa.sw.OUT64 = h->q;
      pa.sw.stash = h->stash32;
    }
    pa.sw.v_stride = h->n;
    pa.sw.out_stride = h->n;
    pa.sw.stash_stride = h->p;
    pa.n = h->n;
    pa.M = M;
    pa.k = h->k;
    pa.kmax = kmax;
    pa.x = h->x;
    pa.r = h->r;
    pa.z = h->z;
    pa.p = h->pv;
    pa.q = h->q;
    pa.S = static_cast<const TS*>(h->pgrid.one.S);
    pa.c = h->cv;
    pa.sc = h->sc;
    pa.acc = h->acc;
    pa.active = h->active;
    pa.nactive = h->nactive;
    pa.tol = tol;
    pa.etol = h->pgrid.one.etol;
    pa.maxit = maxit;
    pa.fixed = fixed;
    pa.use_lmp = lmp;
    pa.pacc = h->pacc;
    pa.W = reinterpret_cast<TS*>(h->Wp);
    // phases: the main tiling while many members are active, then the
    // convergence tail's tilings (eda_autotune), each launch leaving early
    // once the active count falls to the next level whose tiling differs
    const std::vector<eda_handle::TailPlan>& tails = h->tail[sweep64 ? 0 : 1];
    if (!tails.empty() && !h->brk) CU(h, dalloc(h, &h->brk, 1));
    const bool traced = h->trace_on;
    for (int phase = 0;; ++phase) {
      int nact = M;
      if (!tails.empty()) {
        int rc = read_flag(h, h->nactive, &nact);
        if (rc) return rc;
        if (nact <= 0) break;
      } else if (phase > 0) {
        break;
      }
      // the tiling for nact active members: the last level at or above it
      int li = -1;
      for (int i = 0; i < (int)tails.size(); ++i)
        if (tails[i].level >= nact) li = i;
      const SweepPlan& pl = li < 0 ? gp : tails[li].plan;
      const int* tab = li < 0 ? (sweep64 ? (h->tab64_ok ? h->tab64 : nullptr) : (h->tab32_ok ? h->tab32 : nullptr))
                              : tails[li].tab;
      int below = -1;  // leave when at most `below` members remain (-1: run to the end)
      for (int i = li + 1; i < (int)tails.size(); ++i) {
        const SweepPlan& q = tails[i].plan;
        if (q.CS != pl.CS || q.K != pl.K || q.A != pl.A || q.C != pl.C) {
          below = tails[i].level;
          break;
        }
      }
      if (phase > 0) {
        CU(h, cudaMemsetAsync(h->pacc, 0, (size_t)M * sizeof(eda::PersistAcc), h->st));
        CU(h, cudaMemsetAsync(h->Wp, 0, (size_t)2 * M * kmax * sizeof(TS), h->st));
      }
      if (h->brk) CU(h, cudaMemsetAsync(h->brk, 0, sizeof(int), h->st));
      pa.sw.obs_tab = tab;
      pa.exit_below = below;
      pa.brk = below >= 0 ? h->brk : nullptr;
      if (traced) {
        // every persistent launch is traced: its duration, and the columns its
        // sweeps computed (the member iterations it ran)
        rc = trace_begin(h, sweep64 ? 0 : 1, nullptr, 0);
        if (rc) return rc;
        eda::count_launch();
        iters_delta_kernel<<<1, 256, 0, h->st>>>(h->trace_cols + (sweep64 ? 0 : 1), h->sc, M, -1);
      }
      CU(h, eda::launch_pcg_persist<TS>(pa, pl, h->st));
      if (traced) {
        rc = trace_end(h);
        if (rc) return rc;
        eda::count_launch();
        iters_delta_kernel<<<1, 256, 0, h->st>>>(h->trace_cols + (sweep64 ? 0 : 1), h->sc, M, 1);
      }
      if (env_int("EDA_VERBOSE", 0) > 1)
        std::fprintf(stderr, "persistent PCG phase %d: %d active, CS=%d A=%d K=%d, leaves at %d\n", phase, nact,
                     pl.CS, pl.A, pl.K, below);
      if (below < 0) break;
    }
    CU(h, cudaStreamSynchronize(h->st));
    *it_done = it0 + maxit;
    return EDA_OK;
  }
  constexpr int R = eda_handle::kRing;
  // every member stops at convergence or at its own maxit-th iteration, so
  // no loop needs more than maxit iterations
  int it = it0;
  while (it - it0 < maxit) {
    const int par = (it - it0) & 1;
    ++it;
    int rc;
    if (lm.split) {
      // q^ = U H U p^ (U symmetric); the sweep's epilogue adds
      // (U p^).(H U p^) = p^.q^ to the accumulators
      rc = lmp_apply_dev(h, 1, kind, M, h->pv, h->tbuf, h->active);
      if (rc) return rc;
      rc = hvp_dev(h, h->cols, M, h->tbuf, h->q, 1, sweep64, h->active, reinterpret_cast<double*>(h->acc));
      if (rc) return rc;
      rc = lmp_apply_dev(h, 1, kind, M, h->q, h->q, h->active);
    } else {
      rc = hvp_dev(h, h->cols, M, h->pv, h->q, 1, sweep64, h->active, reinterpret_cast<double*>(h->acc));
    }
    if (rc) return rc;
    CU(h, eda::pcg2_update<TS>(h->pgrid, kmax, M, h->pv, h->q, h->x, h->r, h->sc, h->acc,
                               h->active, Wk, par, 1, lmp, h->nactive, h->st));
    if (replace_every > 0 && (it - it0) % replace_every == 0) {
      // residual replacement: the recurrence residual gives way to the FP64
      // true residual b - (I + A) x, and the projections follow it; CG goes
      // on with the same direction
      rc = hvp_dev(h, h->cols, M, h->x, h->q, 1, true, h->active);
      if (rc) return rc;
      CU(h, eda::pcg2_replace(h->pgrid, M, h->b, h->q, h->r, h->acc, M, h->active, h->st));
      CU(h, cudaMemsetAsync(Wk, 0, (size_t)M * kmax * sizeof(TS), h->st));
      CU(h, eda::pcg2_update<TS>(h->pgrid, kmax, M, h->pv, h->q, h->x, h->r, h->sc, h->acc,
                                 h->active, Wk, par, 0, lmp, h->nactive, h->st));
    }
    if (zext) {
      rc = lmp_apply_dev(h, 0, 1, M, h->r, h->z, h->active);
      if (rc) return rc;
    }
    CU(h, eda::pcg2_precond<TS>(h->pgrid, kmax, M, h->r, h->z, h->pv, h->sc, h->acc, h->active,
                                Wk, par, tol, maxit, fixed, lmp, 0, h->nactive, h->st, zext ? h->z : nullptr));
    const int slot = it % R;
    CU(h, eda::pcg2_dir<TS>(h->pgrid, kmax, M, h->z, h->pv, h->sc, h->acc, h->active, Wk, par,
                            h->st, h->nactive, h->hring + slot));
    CU(h, cudaEventRecord(h->ring_ev[slot], h->st));
    if (it - it0 >= R) {
      const int old = (it - R + 1) % R;
      CU(h, cudaEventSynchronize(h->ring_ev[old]));
      if (h->hring[old] == 0) break;
    }
  }
  CU(h, cudaStreamSynchronize(h->st));
  *it_done = it;
  return EDA_OK;
}

int pcg_loop(eda_handle* h, double tol, int maxit, int it0, bool use_lmp, int* it_done, bool sweep64,
             int replace_every = 0, LoopMode lm = LoopMode{}) {
  // the LMP arithmetic follows the sweeps: FP64, or FP32 with the FP32 copy of S
  if (sweep64) return pcg_loop_t<double>(h, tol, maxit, it0, use_lmp, it_done, true, 0, lm);
  return pcg_loop_t<float>(h, tol, maxit, it0, use_lmp, it_done, false, replace_every, lm);
}

}  // namespace

namespace {

// Options of one batched solve (eda_solve; eda_solve_batch fills tol, maxit,
// use_lmp and x0 only).
struct SolveOpts {
  double tol = 0.0, etol = 0.0;
  int maxit = 0, use_lmp = 0, split = 0, lmp_kind = 0;
  const double* x0 = nullptr;
  double* cost = nullptr;
};

int solve_impl(eda_handle* h, const SolveOpts& o, double* dz_out, int* iters_out, double* relres_out,
               double* errb_out, int* status_out) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return fail(h, EDA_ERR_STATE, "solve before eda_set_trajectory");
  if (o.use_lmp && !h->have_lmp) return fail(h, EDA_ERR_STATE, "solve with use_lmp before eda_build_lmp");
  if (!dz_out || o.maxit < 0 || !(o.tol >= 0.0) || !(o.etol >= 0.0))
    return fail(h, EDA_ERR_INVALID, "solve: invalid argument (dz_out NULL, maxit < 0 or a negative tolerance)");
  if (o.lmp_kind != 0 && o.lmp_kind != 1) return fail(h, EDA_ERR_INVALID, "solve: lmp_kind must be 0 or 1");
  if (o.lmp_kind == 1 && h->k > 128) return fail(h, EDA_ERR_INVALID, "solve: the tensor-core LMP takes k <= 128");
  if (o.split != 0) {
    if (!o.use_lmp) return fail(h, EDA_ERR_INVALID, "solve: the split preconditioner needs use_lmp");
    if (h->precision != EDA_FP64) return fail(h, EDA_ERR_INVALID, "solve: the split preconditioner is FP64 only");
    if (o.etol > 0.0) return fail(h, EDA_ERR_INVALID, "solve: err_tol is not available with the split preconditioner");
    // an error e in U v reaches H's leading eigenvalues before U damps them
    // again, so the split iteration needs an LMP accurate to working precision
    if (o.lmp_kind != 0) return fail(h, EDA_ERR_INVALID, "solve: the split preconditioner takes lmp_kind 0");
  }
  const int n = h->n, M = h->M;
  const size_t vb = (size_t)M * n * sizeof(double);
  const LoopMode lm{o.split != 0, o.use_lmp && o.lmp_kind == 1};
  if (lm.tc && h->tc_timeout) CU(h, cudaMemsetAsync(h->tc_timeout, 0, sizeof(int), h->st));
  const long long jstride = (long long)o.maxit + 1;
  In ix0;
  CU(h, ix0.init(o.x0, vb, h->st));
  Out ocost;
  CU(h, ocost.init(o.cost, o.cost ? (size_t)M * jstride * sizeof(double) : 0, h->st));
  // the solve's options travel with the problem to the PCG kernels
  h->pgrid.one.etol = o.etol;
  h->pgrid.one.b = h->b;
  h->pgrid.one.jhist = static_cast<double*>(ocost.dev);
  h->pgrid.one.jstride = (int)jstride;
  struct Reset {  // the handle's other solves run without them
    eda_handle* h;
    ~Reset() {
      h->pgrid.one.etol = 0.0;
      h->pgrid.one.jhist = nullptr;
      h->pgrid.one.b = h->b;
    }
  } reset{h};
  CU(h, cudaMemsetAsync(h->nactive, 0, sizeof(int), h->st));
  const double* bsys = h->b;  // right-hand side of the system CG runs on
  if (lm.split) {
    // CG on U H U y = U b (U = U_theta, Section 3.1, Eq. (lmp)); x = U y at
    // the end.  b^ = U b; from x0: y0 = U^{-1} x0 and r^0 = U (b - H x0)
    if (!h->bh) CU(h, dalloc(h, &h->bh, (size_t)M * n));
    if (!h->tbuf) CU(h, dalloc(h, &h->tbuf, (size_t)M * n));
    const int kind = o.lmp_kind;
    int rc = lmp_apply_dev(h, 1, kind, M, h->b, h->bh, nullptr);
    if (rc) return rc;
    bsys = h->bh;
    h->pgrid.one.b = h->bh;  // the cost record: J(U y) = -y^T (b^ + r^) / 2
    if (o.x0) {
      rc = hvp_dev(h, h->cols, M, static_cast<const double*>(ix0.dev), h->q, 1, true, nullptr);
      if (rc) return rc;
      eda::count_launch();
      sub_kernel<double><<<grid_for((long long)M * n), 256, 0, h->st>>>((long long)M * n, h->b, h->q, h->tbuf);
      CU(h, cudaGetLastError());
      rc = lmp_apply_dev(h, 1, kind, M, h->tbuf, h->r, nullptr);
      if (rc) return rc;
      rc = lmp_apply_dev(h, 2, kind, M, static_cast<const double*>(ix0.dev), h->x, nullptr);
      if (rc) return rc;
    } else {
      CU(h, cudaMemsetAsync(h->x, 0, vb, h->st));
      CU(h, cudaMemcpyAsync(h->r, h->bh, vb, cudaMemcpyDeviceToDevice, h->st));
    }
  } else if (o.x0) {
    // x = x0, r = b - H x0: with the sweeps of the handle's precision (in
    // EDA_MIXED the FP64 true residual at the end checks the result)
    CU(h, cudaMemcpyAsync(h->x, ix0.dev, vb, cudaMemcpyDeviceToDevice, h->st));
    int rc = hvp_dev(h, h->cols, M, h->x, h->q, 1, h->precision == EDA_FP64, nullptr);
    if (rc) return rc;
    eda::count_launch();
    sub_kernel<double><<<grid_for((long long)M * n), 256, 0, h->st>>>((long long)M * n, h->b, h->q, h->r);
  } else {
    CU(h, cudaMemsetAsync(h->x, 0, vb, h->st));
    CU(h, cudaMemcpyAsync(h->r, h->b, vb, cudaMemcpyDeviceToDevice, h->st));
  }
  CU(h, cudaGetLastError());
  if (o.cost) {
    // NaN (all bits set) where no iterate is recorded; J(x0) first
    CU(h, cudaMemsetAsync(ocost.dev, 0xff, (size_t)M * jstride * sizeof(double), h->st));
    eda::count_launch();
    cost0_kernel<<<M, 256, 0, h->st>>>(n, h->x, bsys, h->r, static_cast<double*>(ocost.dev), jstride);
    CU(h, cudaGetLastError());
  }
  CU(h, eda::pcg_start<double>(n, M, bsys, h->r, h->sc, h->active, o.tol, h->nactive, h->st));
  const bool lmp = o.use_lmp != 0;
  const int maxit = o.maxit;
  const double tol = o.tol, etol = o.etol;
  int it = 0;
  if (lm.split) {
    int rc = pcg_loop(h, tol, maxit, 0, lmp, &it, true, 0, lm);
    if (rc) return rc;
    rc = lmp_apply_dev(h, 1, o.lmp_kind, M, h->x, h->x, nullptr);  // x = U y
    if (rc) return rc;
    if (errb_out != nullptr) {
      // the certified bound of the mapped solution (no further rounds: the
      // stopping test of the split iteration is on U r)
      rc = hvp_dev(h, h->cols, M, h->x, h->q, 1, true, nullptr);
      if (rc) return rc;
      CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
      CU(h, cudaMemsetAsync(h->active, 0, (size_t)M * sizeof(int), h->st));
      eda::count_launch(2);
      bnorm_kernel<<<M, 256, 0, h->st>>>(n, h->b, h->sc);
      true_res_kernel<<<M, 256, 0, h->st>>>(n, h->b, h->q, h->x, nullptr, h->r, h->sc, h->active, 0.0, 0.0,
                                           h->nactive, h->dstatus, 0.0, maxit);
      CU(h, cudaGetLastError());
    }
  } else if (h->precision == EDA_FP64) {
    int rc = pcg_loop(h, tol, maxit, 0, lmp, &it, true, 0, lm);
    if (rc) return rc;
    // with a certified bound asked for (as a criterion or an output): the
    // FP64 true residual at exit, and further rounds for members whose
    // true bound misses err_tol (the recurrence residual drifts from it)
    if (etol > 0.0 || errb_out != nullptr) {
      for (int round = 0; round < 64; ++round) {
        rc = hvp_dev(h, h->cols, M, h->x, h->q, 1, true, nullptr);
        if (rc) return rc;
        CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
        eda::count_launch();
        true_res_kernel<<<M, 256, 0, h->st>>>(n, h->b, h->q, h->x, nullptr, h->r, h->sc, h->active, tol, etol,
                                             h->nactive, h->dstatus, 0.0, maxit);
        CU(h, cudaGetLastError());
        int need = 0;
        rc = read_flag(h, h->dstatus, &need);
        if (rc) return rc;
        if (need == 0) break;
        rc = pcg_loop(h, tol, maxit, it, lmp, &it, true, 0, lm);
        if (rc) return rc;
      }
    }
  } else {
    // FP32 sweeps and FP32 LMP arithmetic; CG vectors, scalars and x in FP64.
    // Iterative refinement: every inner PCG reduces its own residual by tau,
    // then the FP64 true residual b - (I + A) x restarts the members that
    // miss a requested criterion.  EDA_MIXED_REPLACE = r > 0 instead
    // replaces the recurrence residual by the FP64 true one every r
    // iterations without a restart; on the batched workload that needs as
    // many iterations and costs the extra FP64 sweeps, so restarts are the
    // default.
    const char* taus = std::getenv("EDA_MIXED_INNER_TOL");
    const double tau = (taus && *taus) ? std::atof(taus) : 1e-3;
    const int rep = env_int("EDA_MIXED_REPLACE", 0);
    const bool crit = tol > 0.0 || etol > 0.0;
    if (rep <= 0 && crit && tau > 0.0) {
      eda::count_launch();
      set_tolm_kernel<<<1, 128, 0, h->st>>>(M, h->sc, tol, etol, tau);
      CU(h, cudaGetLastError());
    }
    int rc = pcg_loop(h, tol, maxit, 0, lmp, &it, false, rep, lm);
    if (rc) return rc;
    // FP64 residual replacement: true residual b - H x with FP64 sweeps;
    // members whose true residual misses a criterion restart from it.
    for (int round = 0; round < 64; ++round) {
      rc = hvp_dev(h, h->cols, M, h->x, h->q, 1, true, nullptr);
      if (rc) return rc;
      CU(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
      eda::count_launch();
      true_res_kernel<<<M, 256, 0, h->st>>>(n, h->b, h->q, h->x, nullptr, h->r, h->sc, h->active, tol, etol,
                                           h->nactive, h->dstatus, tau > 0.0 ? tau : 0.0, maxit);
      CU(h, cudaGetLastError());
      int need = 0;
      rc = read_flag(h, h->dstatus, &need);
      if (rc) return rc;
      if (need == 0 || !crit) break;
      rc = pcg_loop(h, tol, maxit, it, lmp, &it, false, rep, lm);
      if (rc) return rc;
    }
  }
  Out odz, oit, orr, ost, oeb;
  CU(h, odz.init(dz_out, vb, h->st));
  CU(h, oit.init(iters_out, (size_t)M * sizeof(int), h->st));
  CU(h, orr.init(relres_out, (size_t)M * sizeof(double), h->st));
  CU(h, ost.init(status_out, (size_t)M * sizeof(int), h->st));
  CU(h, oeb.init(errb_out, (size_t)M * sizeof(double), h->st));
  CU(h, cudaMemcpyAsync(odz.dev, h->x, vb, cudaMemcpyDeviceToDevice, h->st));
  eda::count_launch();
  export_kernel<<<1, 256, 0, h->st>>>(M, h->sc, (int*)oit.dev, (double*)orr.dev, (int*)ost.dev,
                                      (double*)oeb.dev);
  CU(h, cudaGetLastError());
  CU(h, odz.finish());
  CU(h, oit.finish());
  CU(h, orr.finish());
  CU(h, ost.finish());
  CU(h, oeb.finish());
  CU(h, ocost.finish());
  if (odz.host || oit.host || orr.host || ost.host || oeb.host || ocost.host) CU(h, cudaStreamSynchronize(h->st));
  if (lm.tc) return check_tc_timeout(h);
  return EDA_OK;
}

}  // namespace

extern "C" {

EDA_API int eda_solve_batch(eda_handle* h, double tol, int maxit, const double* x0, int use_lmp, double* dz_out,
                            int* iters_out, double* relres_out, int* status_out) {
  SolveOpts o;
  o.tol = tol;
  o.maxit = maxit;
  o.use_lmp = use_lmp;
  o.x0 = x0;
  return solve_impl(h, o, dz_out, iters_out, relres_out, nullptr, status_out);
}

EDA_API int eda_lmp_apply(eda_handle* h, int which, int kind, int ncol, const double* R, double* Z) {
  if (!h) return fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_lmp) return fail(h, EDA_ERR_STATE, "eda_lmp_apply before eda_build_lmp / eda_set_lmp");
  if (which < 0 || which > 2 || kind < 0 || kind > 1 || ncol < 0 || (ncol > 0 && (!R || !Z)))
    return fail(h, EDA_ERR_INVALID, "eda_lmp_apply: invalid argument");
  if (kind == 1 && h->k > 128) return fail(h, EDA_ERR_INVALID, "eda_lmp_apply: the tensor-core LMP takes k <= 128");
  if (ncol == 0) return EDA_OK;
  const size_t bytes = (size_t)ncol * h->n * sizeof(double);
  In ir;
  Out oz;
  CU(h, ir.init(R, bytes, h->st));
  CU(h, oz.init(Z, bytes, h->st));
  if (kind == 1 && h->tc_timeout) CU(h, cudaMemsetAsync(h->tc_timeout, 0, sizeof(int), h->st));
  int rc = lmp_apply_dev(h, which, kind, ncol, static_cast<const double*>(ir.dev), static_cast<double*>(oz.dev),
                         nullptr);
  if (rc) return rc;
  CU(h, oz.finish());
  if (oz.host) CU(h, cudaStreamSynchronize(h->st));
  if (kind == 1) return check_tc_timeout(h);
  return EDA_OK;
}

EDA_API int eda_solve(eda_handle* h, const eda_solve_opts* opts, double* dz_out, int* iters_out,
                      double* relres_out, double* err_bound_out, int* status_out) {
  if (!opts) return fail(h, EDA_ERR_INVALID, "eda_solve: opts is NULL");
  SolveOpts o;
  o.tol = opts->tol;
  o.etol = opts->err_tol;
  o.maxit = opts->maxit;
  o.use_lmp = opts->use_lmp;
  o.split = opts->split;
  o.lmp_kind = opts->lmp_kind;
  o.x0 = opts->x0;
  o.cost = opts->cost_out;
  return solve_impl(h, o, dz_out, iters_out, relres_out, err_bound_out, status_out);
}

}  // extern "C"
