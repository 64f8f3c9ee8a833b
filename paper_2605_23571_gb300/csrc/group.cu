// Uneven batching: many independent EDA problems (different n, window length,
// member count, observation network and B) solved together.  Every sweep of
// the group -- all members of all problems in the PCG, all sketch columns of
// all problems -- runs as one launch per thread-block shape ("bucket"), with
// per-problem tilings carried by the work items.  The PCG runs as one
// persistent launch per bucket whose clusters take (problem, member) items
// from a device-side queue, the buckets on concurrent streams, the whole
// solve phase captured once in a CUDA graph and replayed; without the
// persistent kernel (EDA_PERSIST=0), one PCG iteration of the whole group is
// a captured graph replayed until every member has converged.  Tilings
// (tile shape and refresh period per problem) are chosen by the group
// autotuner.  Not in the paper: the paper solves one EDA at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "handle.h"

using eda::SweepItem;
using eda::SweepProb;

namespace {

struct Bucket {
  int CS = 1, A = 0, wmax = 0, K = 4;
  size_t smem = 0;
  std::vector<int> probs;          // problems in this bucket
  std::vector<SweepItem> items;    // current work items
  SweepItem* d_items = nullptr;
  int cap = 0;
};

}  // namespace

struct eda_group {
  std::vector<eda_handle*> hs;
  cudaStream_t st = nullptr;   // the group's own stream (graph capture needs a non-legacy stream)
  cudaStream_t hst = nullptr;  // the handles' stream
  cudaEvent_t join = nullptr;
  int prec = EDA_FP64;
  int P = 0, T = 0;
  std::string err;
  // items of the PCG: (problem, member), concatenated member vectors
  std::vector<int> item_prob, item_member, item_n;
  std::vector<long long> item_off, item_soff;
  int* d_n_of = nullptr;
  long long* d_off_of = nullptr;
  const double** d_S_of = nullptr;
  const float** d_S32_of = nullptr;
  const double** d_c_of = nullptr;
  int* d_k_of = nullptr;
  int kmax = 0;
  int mmax = 0;  // largest member count of the problems
  long long vtot = 0, stot = 0;
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double* stash64 = nullptr;
  float* stash32 = nullptr;
  PcgScalars* sc = nullptr;
  eda::PcgAcc* acc = nullptr;     // per-item accumulators of an iteration
  eda::PersistAcc* pacc = nullptr;  // persistent PCG: per-item accumulators by parity
  double* Wp = nullptr;             // persistent PCG: projections [2][T][kmax] (8 bytes an entry)
  int* queue = nullptr;             // persistent PCG: one work-queue head per bucket
  std::vector<cudaStream_t> bstreams;  // persistent PCG: one stream per bucket (they run concurrently)
  std::vector<cudaEvent_t> bevents;
  double* Wk = nullptr;           // T x max(kmax,1) LMP projections
  eda::PcgTask* tasks = nullptr;  // row chunks of every problem
  int ntasks = 0;
  eda::PcgProb* probs = nullptr;  // per problem: sizes, items, S (of the group's precision), c
  eda::PcgGrid pgrid{};           // the two tables above as the PCG kernels' grid
  int* active = nullptr;
  int* nactive = nullptr;
  int* dflag = nullptr;
  int* hring = nullptr;
  cudaEvent_t ev[4] = {};
  // per-problem sweep descriptors (FP64 and FP32 tilings) and their buckets
  SweepProb<double>* d_prob64 = nullptr;
  SweepProb<float>* d_prob32 = nullptr;
  std::vector<SweepProb<double>> prob64;
  std::vector<SweepProb<float>> prob32;
  std::vector<int*> tabs;
  std::vector<Bucket> b64, b32;
  // sketch: concatenated Phi / Y of all problems
  long long ktot = 0;
  std::vector<long long> sk_off;
  double *Phi = nullptr, *Y = nullptr;
  double* sk_stash64 = nullptr;
  float* sk_stash32 = nullptr;
  // captured PCG iteration
  cudaGraphExec_t gexec = nullptr;
  // the persistent solve phase (memsets, every bucket's launch on its stream,
  // the join) captured once and replayed while its signature holds
  cudaGraphExec_t pexec = nullptr;
  std::vector<long long> psig;
  int g_key = -1;
  double g_tol = -1.0;
  int g_maxit = -1;
  std::vector<void*> allocs;
};

namespace {

int gfail(eda_group* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  return eda::fail(nullptr, code, msg);
}

#define GCU(g, ...)                                                                                \
  do {                                                                                             \
    cudaError_t e__ = (__VA_ARGS__);                                                               \
    if (e__ != cudaSuccess)                                                                        \
      return gfail((g), EDA_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__)); \
  } while (0)

template <typename T>
cudaError_t galloc(eda_group* g, T** ptr, size_t count) {
  cudaError_t e = cudaMalloc((void**)ptr, (count ? count : 1) * sizeof(T));
  if (e == cudaSuccess) g->allocs.push_back((void*)*ptr);
  return e;
}

// The group works on its own stream, ordered after / before the handles'.
int enter(eda_group* g) {
  GCU(g, cudaEventRecord(g->join, g->hst));
  GCU(g, cudaStreamWaitEvent(g->st, g->join, 0));
  return EDA_OK;
}
int leave(eda_group* g) {
  GCU(g, cudaEventRecord(g->join, g->st));
  GCU(g, cudaStreamWaitEvent(g->hst, g->join, 0));
  return EDA_OK;
}

// ---------------------------------------------------------------- kernels
__global__ void g_true_res_kernel(const int* n_of, const long long* off_of, const double* b, const double* hx,
                                  double* r, PcgScalars* sc, int* active, double tol, int* nactive, int* need,
                                  double tau, int maxit) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const int n = n_of[j];
  const long long off = off_of[j];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double rv = b[off + i] - hx[off + i];
    r[off + i] = rv;
    s += rv * rv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    const double bn = sc[j].bnorm;
    const double rel = bn > 0.0 ? sqrt(t) / bn : 0.0;
    sc[j].relres = rel;
    const bool ok = (bn == 0.0) || (rel <= tol);
    if (sc[j].status == EDA_CONVERGED && !ok) {
      sc[j].status = EDA_MAXIT;
      if (sc[j].iters < maxit) {  // next refinement round, within the member's budget
        sc[j].tolm = fmax(tol, tau * rel);
        active[j] = 1;
        atomicAdd(nactive, 1);
        atomicAdd(need, 1);
      }
    }
  }
}

__global__ void g_set_tolm_kernel(int T, PcgScalars* sc, double tol, double tau) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x)
    sc[j].tolm = fmax(tol, tau * sc[j].relres);
}

__global__ void g_export_kernel(int T, const PcgScalars* sc, int* iters, double* relres, int* status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x) {
    if (iters) iters[j] = sc[j].iters;
    if (relres) relres[j] = sc[j].relres;
    if (status) status[j] = sc[j].status;
  }
}

__global__ void g_gamma_kernel(int n, int ell, const double* b, double* Phi) {
  const long long total = (long long)ell * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    Phi[i] = b[(i / n + 1) * n + (i % n)] - b[i % n];
}

// ---------------------------------------------------------------- planning
template <typename T>
SweepProb<T> make_prob(eda_handle* h, const SweepPlan& pl, int* tab) {
  SweepProb<T> P{};
  P.n = h->n;
  P.N = h->N;
  P.p = h->p;
  P.w = h->w;
  P.nos = h->nos;
  P.Ttile = pl.Ttile;
  P.HL = pl.HL;
  P.E = pl.E;
  P.K = pl.K;
  P.A = pl.A;
  P.F = (T)h->F;
  P.dt = (T)h->dt;
  P.traj_mstride = (long long)(h->N + 1) * h->n;
  P.obs_of_t = h->obs_of_t;
  P.obs_ptr = h->obs_ptr;
  P.obs_idx = h->obs_idx;
  P.obs_tab = tab;
  if constexpr (sizeof(T) == 8) {
    P.traj = h->traj;
    P.rinv = h->rinv;
    P.bcoef = h->bcoef;
  } else {
    P.traj = h->traj32;
    P.rinv = h->rinv32;
    P.bcoef = h->bcoef32;
  }
  return P;
}

// Plans every problem for one precision with refresh period K (per bucket
// later), groups problems into buckets by cluster size and thread count.
// Tilings and buckets of every problem: halo refresh period Kp[pi] and a
// tile shape of mult[pi] (1 or 2) times the fewest CTAs per member that fit
// (mult empty: 1), falling back to the fewest where the wider shape does not
// fit.
int plan_group(eda_group* g, bool fp64, const std::vector<int>& Kp, const std::vector<int>& mult = {}) {
  const int eb = fp64 ? 8 : 4;
  std::vector<Bucket>& bs = fp64 ? g->b64 : g->b32;
  std::map<std::pair<int, int>, int> key2b;
  std::vector<Bucket> nb;
  std::vector<SweepPlan> plans(g->P);
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    SweepPlan pl;
    bool ok = false;
    for (int CS = 1; CS <= 16 && !ok; ++CS) ok = eda::plan_sweep_exact(h->n, eb, h->w, CS, Kp[pi], &pl);
    if (ok && !mult.empty() && mult[pi] > 1) {
      SweepPlan wide;
      const int cs2 = pl.CS * mult[pi];
      if (cs2 <= 16 && eda::plan_sweep_exact(h->n, eb, h->w, cs2, Kp[pi], &wide) && wide.HL <= h->n) pl = wide;
    }
    if (!ok && !eda::plan_sweep(h->n, eb, h->w, 1, 0, &pl))
      return gfail(g, EDA_ERR_INVALID, "group: a problem does not fit the sweep tiling");
    if (pl.ml)
      return gfail(g, EDA_ERR_INVALID,
                   "group: problem " + std::to_string(pi) + " (n = " + std::to_string(h->n) +
                       ") needs multi-launch sweeps; solve it on its own handle");
    plans[pi] = pl;
    int Ab = 32;
    while (Ab < pl.A) Ab *= 2;
    const auto key = std::make_pair(pl.CS, Ab);
    if (!key2b.count(key)) {
      key2b[key] = (int)nb.size();
      Bucket b;
      b.CS = pl.CS;
      b.A = Ab;
      nb.push_back(b);
    }
    Bucket& b = nb[key2b[key]];
    b.probs.push_back(pi);
    b.wmax = std::max(b.wmax, h->w);
    b.K = pl.K;
  }
  // observation tables and descriptors
  std::vector<SweepProb<double>> P64;
  std::vector<SweepProb<float>> P32;
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    std::vector<int> tab((size_t)plans[pi].CS * h->nos * 8);
    bool usable = false;
    eda::obs_table(plans[pi], h->n, h->nos, h->h_obs_ptr.data(), h->h_obs_idx.data(), tab.data(), &usable);
    int* dt = nullptr;
    if (usable) {
      GCU(g, cudaMalloc((void**)&dt, tab.size() * sizeof(int)));
      g->tabs.push_back(dt);
      GCU(g, cudaMemcpy(dt, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (fp64)
      P64.push_back(make_prob<double>(h, plans[pi], dt));
    else
      P32.push_back(make_prob<float>(h, plans[pi], dt));
  }
  for (Bucket& b : nb) b.smem = eda::sweep_smem_bytes(b.A, fp64 ? 4 : 8, b.wmax, eb);
  if (fp64) {
    g->prob64 = P64;
    if (!g->d_prob64) GCU(g, galloc(g, &g->d_prob64, g->P));
    GCU(g, cudaMemcpy(g->d_prob64, P64.data(), P64.size() * sizeof(P64[0]), cudaMemcpyHostToDevice));
  } else {
    g->prob32 = P32;
    if (!g->d_prob32) GCU(g, galloc(g, &g->d_prob32, g->P));
    GCU(g, cudaMemcpy(g->d_prob32, P32.data(), P32.size() * sizeof(P32[0]), cudaMemcpyHostToDevice));
  }
  for (Bucket& b : bs)
    if (b.d_items) cudaFree(b.d_items);
  bs = nb;
  return EDA_OK;
}

// Work items of the PCG products (every member of every problem) or of the
// sketch (every column of every problem on its control trajectory).
int set_items(eda_group* g, bool fp64, bool sketch) {
  std::vector<Bucket>& bs = fp64 ? g->b64 : g->b32;
  for (Bucket& b : bs) {
    b.items.clear();
    for (int pi : b.probs) {
      eda_handle* h = g->hs[pi];
      if (sketch) {
        for (int c = 0; c < h->ell; ++c) {
          SweepItem it{};
          it.prob = pi;
          it.member = 0;
          it.flag = -1;
          it.voff = g->sk_off[pi] + (long long)c * h->n;
          it.soff = 0;  // filled below
          b.items.push_back(it);
        }
      } else {
        for (int j = 0; j < g->T; ++j) {
          if (g->item_prob[j] != pi) continue;
          SweepItem it{};
          it.prob = pi;
          it.member = g->item_member[j];
          it.flag = j;
          it.voff = g->item_off[j];
          it.soff = g->item_soff[j];
          b.items.push_back(it);
        }
      }
    }
    // largest problems first: the block scheduler then balances the tail
    std::stable_sort(b.items.begin(), b.items.end(), [&](const SweepItem& u, const SweepItem& v) {
      const eda_handle* hu = g->hs[u.prob];
      const eda_handle* hv = g->hs[v.prob];
      return (long long)hu->n * hu->N > (long long)hv->n * hv->N;
    });
    if ((int)b.items.size() > b.cap) {
      if (b.d_items) cudaFree(b.d_items);
      b.d_items = nullptr;
      b.cap = (int)b.items.size();
      GCU(g, cudaMalloc((void**)&b.d_items, (size_t)std::max(b.cap, 1) * sizeof(SweepItem)));
    }
  }
  if (sketch) {
    // stash offsets of sketch items (one stash per sketch column)
    long long off = 0;
    for (Bucket& b : bs)
      for (SweepItem& it : b.items) {
        it.soff = off;
        off += g->hs[it.prob]->p;
      }
  }
  for (Bucket& b : bs)
    if (!b.items.empty())
      GCU(g, cudaMemcpyAsync(b.d_items, b.items.data(), b.items.size() * sizeof(SweepItem), cudaMemcpyHostToDevice,
                             g->st));
  return EDA_OK;
}

// One launch per bucket: HV = V + A V (ident) or A V for the current items.
int group_sweep(eda_group* g, bool fp64, const double* V, double* HV, int ident, bool sketch,
                double* dot = nullptr) {
  std::vector<Bucket>& bs = fp64 ? g->b64 : g->b32;
  for (Bucket& b : bs) {
    if (b.items.empty()) continue;
    SweepPlan pl{};
    pl.CS = b.CS;
    pl.C = fp64 ? 4 : 8;
    pl.A = b.A;
    pl.E = b.A * pl.C;
    pl.Ttile = 0;
    pl.HL = 0;
    pl.K = b.K;
    pl.smem = b.smem;
    if (fp64) {
      SweepArgs<double> a{};
      a.mode = eda::MODE_HVP;
      a.ncol = (int)b.items.size();
      a.w = b.wmax;
      a.V64 = V;
      a.OUT64 = HV;
      a.stash = sketch ? g->sk_stash64 : g->stash64;
      a.include_identity = ident;
      a.probs = g->d_prob64;
      a.items = b.d_items;
      a.flags = g->active;
      a.dot_out = dot;
      a.dot_stride = eda::kPcgAccStride;
      a.n = 1;
      GCU(g, eda::launch_sweep<double>(a, pl, g->st));
    } else {
      SweepArgs<float> a{};
      a.mode = eda::MODE_HVP;
      a.ncol = (int)b.items.size();
      a.w = b.wmax;
      a.V64 = V;
      a.OUT64 = HV;
      a.stash = sketch ? g->sk_stash32 : g->stash32;
      a.include_identity = ident;
      a.probs = g->d_prob32;
      a.items = b.d_items;
      a.flags = g->active;
      a.dot_out = dot;
      a.dot_stride = eda::kPcgAccStride;
      a.n = 1;
      GCU(g, eda::launch_sweep<float>(a, pl, g->st));
    }
  }
  return EDA_OK;
}

// The work of one PCG iteration of the whole group (iteration parity par):
// the batched sweeps with p.q in their epilogue, then the update, precond and
// dir launches over row chunks of every problem (pcg.h).
template <typename TS>
int group_iteration(eda_group* g, bool sweep64, bool use_lmp, double tol, int maxit, int fixed, int par) {
  const int kmax = std::max(g->kmax, 1);
  const int lmp = use_lmp ? 1 : 0;
  TS* Wk = reinterpret_cast<TS*>(g->Wk);
  int rc = group_sweep(g, sweep64, g->p, g->q, 1, false, reinterpret_cast<double*>(g->acc));
  if (rc) return rc;
  GCU(g, eda::pcg2_update<TS>(g->pgrid, kmax, g->mmax, g->p, g->q, g->x, g->r, g->sc, g->acc, g->active,
                              Wk, par, 1, lmp, g->nactive, g->st));
  GCU(g, eda::pcg2_precond<TS>(g->pgrid, kmax, g->mmax, g->r, g->z, g->p, g->sc, g->acc, g->active, Wk,
                               par, tol, maxit, fixed, lmp, 0, g->nactive, g->st));
  GCU(g, eda::pcg2_dir<TS>(g->pgrid, kmax, g->mmax, g->z, g->p, g->sc, g->acc, g->active, Wk, par,
                           g->st));
  return EDA_OK;
}

// Start of a PCG loop: z = P r, p = z, r.z for the active items.
template <typename TS>
int group_start(eda_group* g, bool use_lmp, double tol, int maxit, int fixed) {
  const int kmax = std::max(g->kmax, 1);
  const int lmp = use_lmp ? 1 : 0;
  TS* Wk = reinterpret_cast<TS*>(g->Wk);
  GCU(g, eda::pcg2_reset(g->acc, g->T, Wk, (size_t)g->T * kmax * sizeof(TS), g->st));
  GCU(g, eda::pcg2_update<TS>(g->pgrid, kmax, g->mmax, g->p, g->q, g->x, g->r, g->sc, g->acc, g->active,
                              Wk, 0, 0, lmp, g->nactive, g->st));
  GCU(g, eda::pcg2_precond<TS>(g->pgrid, kmax, g->mmax, g->r, g->z, g->p, g->sc, g->acc, g->active, Wk,
                               0, tol, maxit, fixed, lmp, 1, g->nactive, g->st));
  // the first update accumulates the projections of r_1 from zero
  GCU(g, cudaMemsetAsync(Wk, 0, (size_t)g->T * kmax * sizeof(TS), g->st));
  return EDA_OK;
}

// The whole PCG loop of the group as one persistent launch per bucket: the
// bucket's clusters take its (problem, member) items, largest problems first,
// from a device-side queue and run each member's PCG to its stop (pcg.h).
template <typename TS>
int group_persist(eda_group* g, bool sweep64, bool use_lmp, double tol, int maxit, int fixed, int* it_io) {
  const int kmax = std::max(g->kmax, 1);
  std::vector<Bucket>& bs = sweep64 ? g->b64 : g->b32;
  if (!g->pacc) GCU(g, galloc(g, &g->pacc, (size_t)g->T));
  if (!g->Wp) GCU(g, galloc(g, &g->Wp, (size_t)2 * g->T * kmax));
  if (!g->queue) GCU(g, galloc(g, &g->queue, (size_t)64));
  // every bucket on its own stream, forked from and joined to the group's
  while (g->bstreams.size() < bs.size()) {
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev2 = nullptr;
    GCU(g, cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    g->bstreams.push_back(st2);
    GCU(g, cudaEventCreateWithFlags(&ev2, cudaEventDisableTiming));
    g->bevents.push_back(ev2);
  }
  // the launches: one persistent PCG per non-empty bucket
  struct Launch {
    eda::PersistArgs<TS> pa;
    SweepPlan pl;
    size_t bucket;
  };
  std::vector<Launch> ls;
  std::vector<long long> sig = {sweep64 ? 1 : 0, use_lmp ? 1 : 0, fixed, maxit, 0};
  std::memcpy(&sig[4], &tol, sizeof(double));
  int qi = 0;
  for (size_t bi = 0; bi < bs.size(); ++bi) {
    const Bucket& b = bs[bi];
    if (b.items.empty()) continue;
    // the between-sweep scratch must fit the bucket's shared memory
    int tmax = 0;
    for (int pi : b.probs) tmax = std::max(tmax, sweep64 ? g->prob64[pi].Ttile : g->prob32[pi].Ttile);
    const size_t scratch = 32 * sizeof(double) + (size_t)(((kmax + 3) & ~3) + tmax) * sizeof(TS);
    if (scratch > b.smem || qi >= 64) return gfail(g, EDA_ERR_INVALID, "group: persistent PCG scratch does not fit");
    Launch L{};
    L.bucket = bi;
    L.pl.CS = b.CS;
    L.pl.C = sweep64 ? 4 : 8;
    L.pl.A = b.A;
    L.pl.E = b.A * L.pl.C;
    L.pl.K = b.K;
    L.pl.smem = b.smem;
    eda::PersistArgs<TS>& pa = L.pa;
    pa.sw.w = b.wmax;
    if constexpr (sizeof(TS) == 8) {
      pa.sw.V = g->p;
      pa.sw.OUT = g->q;
      pa.sw.stash = g->stash64;
      pa.sw.probs = g->d_prob64;
    } else {
      pa.sw.V64 = g->p;
      pa.sw.OUT64 = g->q;
      pa.sw.stash = g->stash32;
      pa.sw.probs = g->d_prob32;
    }
    pa.sw.items = b.d_items;
    pa.sw.flags = g->active;
    pa.sw.n = 1;
    pa.n = 1;
    pa.M = g->T;
    pa.kmax = kmax;
    pa.x = g->x;
    pa.r = g->r;
    pa.z = g->z;
    pa.p = g->p;
    pa.q = g->q;
    pa.sc = g->sc;
    pa.acc = g->acc;
    pa.active = g->active;
    pa.nactive = g->nactive;
    pa.tol = tol;
    pa.maxit = maxit;
    pa.fixed = fixed;
    pa.use_lmp = use_lmp ? 1 : 0;
    pa.pacc = g->pacc;
    pa.W = reinterpret_cast<TS*>(g->Wp);
    pa.items = b.d_items;
    pa.nitems = (int)b.items.size();
    pa.pprobs = g->probs;
    pa.queue = g->queue + qi++;
    ls.push_back(L);
    for (long long v : {(long long)reinterpret_cast<uintptr_t>(b.d_items), (long long)b.items.size(),
                        (long long)b.CS, (long long)b.A, (long long)b.K, (long long)b.smem, (long long)bi})
      sig.push_back(v);
  }
  // EDA_VERBOSE: each bucket's launch timed on its stream (no graph)
  const bool verbose = eda::env_int("EDA_VERBOSE", 0) != 0;
  const bool use_graph = eda::env_int("EDA_GROUP_GRAPH", 1) != 0 && !verbose;
  std::vector<cudaEvent_t> tev;
  auto record = [&]() -> int {
    GCU(g, cudaMemsetAsync(g->pacc, 0, (size_t)g->T * sizeof(eda::PersistAcc), g->st));
    GCU(g, cudaMemsetAsync(g->Wp, 0, (size_t)2 * g->T * kmax * sizeof(double), g->st));
    GCU(g, cudaMemsetAsync(g->queue, 0, (size_t)64 * sizeof(int), g->st));
    GCU(g, cudaEventRecord(g->join, g->st));
    for (const Launch& L : ls) {
      cudaStream_t bst = g->bstreams[L.bucket];
      GCU(g, cudaStreamWaitEvent(bst, g->join, 0));
      if (verbose) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        GCU(g, cudaEventCreate(&e0));
        GCU(g, cudaEventCreate(&e1));
        tev.push_back(e0);
        tev.push_back(e1);
        GCU(g, cudaEventRecord(e0, bst));
      }
      GCU(g, eda::launch_pcg_persist<TS>(L.pa, L.pl, bst));
      if (verbose) GCU(g, cudaEventRecord(tev.back(), bst));
      GCU(g, cudaEventRecord(g->bevents[L.bucket], bst));
      GCU(g, cudaStreamWaitEvent(g->st, g->bevents[L.bucket], 0));
    }
    return EDA_OK;
  };
  if (use_graph) {
    if (g->pexec == nullptr || g->psig != sig) {
      if (g->pexec) {
        cudaGraphExecDestroy(g->pexec);
        g->pexec = nullptr;
      }
      // function attributes and grid sizes are settled outside the capture
      for (const Launch& L : ls) {
        int fit = 0;
        GCU(g, eda::launch_pcg_persist<TS>(L.pa, L.pl, g->st, &fit));
      }
      cudaGraph_t graph;
      GCU(g, cudaStreamBeginCapture(g->st, cudaStreamCaptureModeRelaxed));
      const int rc = record();
      cudaError_t ce = cudaStreamEndCapture(g->st, &graph);
      if (rc) return rc;
      GCU(g, ce);
      ce = cudaGraphInstantiate(&g->pexec, graph, 0);
      cudaGraphDestroy(graph);
      GCU(g, ce);
      g->psig = sig;
    }
    eda::count_launch((int)ls.size());
    GCU(g, cudaGraphLaunch(g->pexec, g->st));
  } else {
    const int rc = record();
    if (rc) return rc;
  }
  GCU(g, cudaStreamSynchronize(g->st));
  if (verbose) {
    for (size_t j = 0; j < ls.size(); ++j) {
      const Bucket& b = bs[ls[j].bucket];
      float ms = 0.f;
      GCU(g, cudaEventElapsedTime(&ms, tev[2 * j], tev[2 * j + 1]));
      long long work = 0;  // member x n x window of the bucket
      for (int pi : b.probs) work += (long long)g->hs[pi]->M * g->hs[pi]->n * g->hs[pi]->N;
      std::fprintf(stderr, "persistent group bucket CS=%d A=%d K=%d problems=%zu items=%zu work=%lld: %.1f ms\n",
                   b.CS, b.A, b.K, b.probs.size(), b.items.size(), work, ms);
      cudaEventDestroy(tev[2 * j]);
      cudaEventDestroy(tev[2 * j + 1]);
    }
  }
  *it_io += maxit;
  return EDA_OK;
}

// PCG iterations of the group from the current (x, r): replay of a graph of
// two iterations (parities 0 and 1) with the active count polled through a
// ring of pinned copies.
template <typename TS>
int group_pcg_loop_t(eda_group* g, bool sweep64, bool use_lmp, double tol, int maxit, int* it_io) {
  const int fixed = tol > 0.0 ? 0 : maxit;
  int rc = group_start<TS>(g, use_lmp, tol, maxit, fixed);
  if (rc) return rc;
  if (maxit >= 1 && eda::env_int("EDA_PERSIST", 1)) return group_persist<TS>(g, sweep64, use_lmp, tol, maxit, fixed, it_io);
  const int key = (sweep64 ? 1 : 0) + (use_lmp ? 2 : 0) + (fixed ? 4 : 0);
  const bool use_graph = eda::env_int("EDA_GROUP_GRAPH", 1) != 0;
  // the graph bakes in tol and maxit as kernel arguments
  if (use_graph && (g->gexec == nullptr || g->g_key != key || g->g_tol != tol || g->g_maxit != maxit)) {
    if (g->gexec) {
      cudaGraphExecDestroy(g->gexec);
      g->gexec = nullptr;
    }
    cudaGraph_t graph;
    GCU(g, cudaStreamBeginCapture(g->st, cudaStreamCaptureModeRelaxed));
    rc = group_iteration<TS>(g, sweep64, use_lmp, tol, maxit, fixed, 0);
    if (!rc) rc = group_iteration<TS>(g, sweep64, use_lmp, tol, maxit, fixed, 1);
    cudaError_t ce = cudaStreamEndCapture(g->st, &graph);
    if (rc) return rc;
    GCU(g, ce);
    GCU(g, cudaGraphInstantiate(&g->gexec, graph, 0));
    cudaGraphDestroy(graph);
    g->g_key = key;
    g->g_tol = tol;
    g->g_maxit = maxit;
  }
  constexpr int R = 4;
  // every member stops at convergence or at its own maxit-th iteration, so
  // no loop needs more than maxit iterations (one more at most: the graph
  // runs iterations in pairs, and a member past its budget is inactive)
  int it = *it_io;
  const int it0 = it;
  int polls = 0;
  while (it - it0 < maxit) {
    if (use_graph) {
      eda::count_launch(2 * (4 + (int)(sweep64 ? g->b64.size() : g->b32.size())));
      GCU(g, cudaGraphLaunch(g->gexec, g->st));
    } else {
      rc = group_iteration<TS>(g, sweep64, use_lmp, tol, maxit, fixed, 0);
      if (!rc) rc = group_iteration<TS>(g, sweep64, use_lmp, tol, maxit, fixed, 1);
      if (rc) return rc;
    }
    it += 2;
    ++polls;
    const int slot = polls % R;
    GCU(g, cudaMemcpyAsync(g->hring + slot, g->nactive, sizeof(int), cudaMemcpyDeviceToHost, g->st));
    GCU(g, cudaEventRecord(g->ev[slot], g->st));
    if (polls >= R) {
      const int old = (polls - R + 1) % R;
      GCU(g, cudaEventSynchronize(g->ev[old]));
      if (g->hring[old] == 0) break;
    }
  }
  GCU(g, cudaStreamSynchronize(g->st));
  *it_io = it;
  return EDA_OK;
}

int group_pcg_loop(eda_group* g, bool sweep64, bool use_lmp, double tol, int maxit, int* it_io) {
  // the LMP arithmetic follows the sweeps: FP64, or FP32 with the FP32 copies of S
  if (sweep64) return group_pcg_loop_t<double>(g, true, use_lmp, tol, maxit, it_io);
  return group_pcg_loop_t<float>(g, false, use_lmp, tol, maxit, it_io);
}

}  // namespace

extern "C" {

EDA_API int eda_group_create(eda_handle* const* handles, int count, eda_group** out) {
  if (!out) return eda::fail(nullptr, EDA_ERR_INVALID, "eda_group_create: out is NULL");
  *out = nullptr;
  if (!handles || count < 1) return eda::fail(nullptr, EDA_ERR_INVALID, "eda_group_create: no handles");
  for (int i = 0; i < count; ++i)
    if (!handles[i]) return eda::fail(nullptr, EDA_ERR_INVALID, "eda_group_create: NULL handle");
  const int prec = handles[0]->precision;
  for (int i = 0; i < count; ++i) {
    if (handles[i]->precision != prec)
      return eda::fail(nullptr, EDA_ERR_INVALID, "eda_group_create: handles must share the precision");
    if (handles[i]->ckpt != 0)
      return eda::fail(nullptr, EDA_ERR_INVALID, "eda_group_create: checkpointed handles are not grouped");
    if (handles[i]->st != handles[0]->st)
      return eda::fail(nullptr, EDA_ERR_INVALID, "eda_group_create: handles must share the stream");
  }
  eda_group* g = new eda_group();
  auto bail = [&](int code) {
    eda_group_destroy(g);
    return code;
  };
  g->hs.assign(handles, handles + count);
  g->hst = handles[0]->st;
  if (cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->join, cudaEventDisableTiming) != cudaSuccess) {
    eda::fail(nullptr, EDA_ERR_CUDA, "eda_group_create: stream/event creation failed");
    return bail(EDA_ERR_CUDA);
  }
  g->prec = prec;
  g->P = count;
  long long voff = 0, soff = 0, koff = 0;
  std::vector<const double*> S_of;
  std::vector<const float*> S32_of;
  std::vector<const double*> c_of;
  std::vector<int> k_of;
  for (int pi = 0; pi < count; ++pi) {
    eda_handle* h = handles[pi];
    for (int m = 0; m < h->M; ++m) {
      g->item_prob.push_back(pi);
      g->item_member.push_back(m);
      g->item_n.push_back(h->n);
      g->item_off.push_back(voff);
      g->item_soff.push_back(soff);
      S_of.push_back(h->k > 0 ? h->S : nullptr);
      S32_of.push_back(h->k > 0 ? h->S32 : nullptr);
      c_of.push_back(h->cv);
      k_of.push_back(h->k);
      g->kmax = std::max(g->kmax, h->k);
      g->mmax = std::max(g->mmax, h->M);
      voff += h->n;
      soff += h->p;
    }
    g->sk_off.push_back(koff);
    koff += (long long)h->ell * h->n;
  }
  g->T = (int)g->item_prob.size();
  g->vtot = voff;
  g->stot = soff;
  g->ktot = koff;
  const int T = g->T;
  if (galloc(g, &g->d_n_of, T) || galloc(g, &g->d_off_of, T) || galloc(g, &g->d_S_of, T) ||
      galloc(g, &g->d_S32_of, T) || galloc(g, &g->d_c_of, T) || galloc(g, &g->d_k_of, T) ||
      galloc(g, &g->b, voff) || galloc(g, &g->x, voff) || galloc(g, &g->r, voff) || galloc(g, &g->z, voff) ||
      galloc(g, &g->p, voff) || galloc(g, &g->q, voff) || galloc(g, &g->stash64, soff) ||
      galloc(g, &g->stash32, soff) || galloc(g, &g->sc, T) || galloc(g, &g->active, T) ||
      galloc(g, &g->nactive, 1) || galloc(g, &g->dflag, 1) || galloc(g, &g->Phi, koff) || galloc(g, &g->Y, koff) ||
      galloc(g, &g->acc, T) || galloc(g, &g->Wk, (long long)T * std::max(g->kmax, 1)) ||
      galloc(g, &g->probs, count)) {
    eda::fail(nullptr, EDA_ERR_CUDA, "eda_group_create: out of device memory");
    return bail(EDA_ERR_CUDA);
  }
  long long skst = 0;
  for (int pi = 0; pi < count; ++pi) skst += (long long)handles[pi]->ell * handles[pi]->p;
  if (galloc(g, &g->sk_stash64, skst) || galloc(g, &g->sk_stash32, skst)) {
    eda::fail(nullptr, EDA_ERR_CUDA, "eda_group_create: out of device memory");
    return bail(EDA_ERR_CUDA);
  }
  cudaError_t e = cudaMemcpy(g->d_n_of, g->item_n.data(), T * sizeof(int), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(g->d_off_of, g->item_off.data(), T * sizeof(long long), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(g->d_S_of, S_of.data(), T * sizeof(void*), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(g->d_S32_of, S32_of.data(), T * sizeof(void*), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(g->d_c_of, c_of.data(), T * sizeof(void*), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(g->d_k_of, k_of.data(), T * sizeof(int), cudaMemcpyHostToDevice);
  {
    // the problems as one PCG batch: row-chunk tasks and per-problem records
    std::vector<eda::PcgProb> pr(count);
    std::vector<int> n_of(count);
    int item = 0;
    for (int pi = 0; pi < count; ++pi) {
      eda_handle* h = handles[pi];
      pr[pi].n = h->n;
      pr[pi].M = h->M;
      pr[pi].k = h->k;
      pr[pi].item0 = item;
      pr[pi].off0 = g->item_off[item];
      pr[pi].S = (h->k > 0) ? ((prec == EDA_MIXED) ? (const void*)h->S32 : (const void*)h->S) : nullptr;
      pr[pi].c = h->cv;
      n_of[pi] = h->n;
      item += h->M;
    }
    std::vector<eda::PcgTask> tasks;
    eda::pcg_tasks(n_of.data(), count, &tasks);
    g->ntasks = (int)tasks.size();
    if (!e) e = galloc(g, &g->tasks, tasks.size());
    if (!e) e = cudaMemcpy(g->tasks, tasks.data(), tasks.size() * sizeof(eda::PcgTask), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(g->probs, pr.data(), pr.size() * sizeof(eda::PcgProb), cudaMemcpyHostToDevice);
    g->pgrid = eda::pcg_tables(g->tasks, g->ntasks, g->probs);
  }
  if (!e) e = cudaMallocHost((void**)&g->hring, 4 * sizeof(int));
  for (int i = 0; i < 4 && !e; ++i) e = cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming);
  if (e) {
    eda::fail(nullptr, EDA_ERR_CUDA, std::string("eda_group_create: ") + cudaGetErrorString(e));
    return bail(EDA_ERR_CUDA);
  }
  std::vector<int> Kp(count);
  for (int pi = 0; pi < count; ++pi) Kp[pi] = (handles[pi]->n <= 512) ? 2 : 4;
  if (plan_group(g, true, Kp) != EDA_OK || set_items(g, true, false) != EDA_OK) return bail(EDA_ERR_INVALID);
  if (prec == EDA_MIXED && (plan_group(g, false, Kp) != EDA_OK || set_items(g, false, false) != EDA_OK))
    return bail(EDA_ERR_INVALID);
  *out = g;
  return EDA_OK;
}

EDA_API int eda_group_destroy(eda_group* g) {
  if (!g) return EDA_OK;
  if (g->st) cudaStreamSynchronize(g->st);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->pexec) cudaGraphExecDestroy(g->pexec);
  for (void* p : g->allocs) cudaFree(p);
  for (int* t : g->tabs) cudaFree(t);
  for (Bucket& b : g->b64)
    if (b.d_items) cudaFree(b.d_items);
  for (Bucket& b : g->b32)
    if (b.d_items) cudaFree(b.d_items);
  if (g->hring) cudaFreeHost(g->hring);
  for (int i = 0; i < 4; ++i)
    if (g->ev[i]) cudaEventDestroy(g->ev[i]);
  if (g->join) cudaEventDestroy(g->join);
  for (cudaEvent_t e : g->bevents) cudaEventDestroy(e);
  for (cudaStream_t st2 : g->bstreams) {
    cudaStreamSynchronize(st2);
    cudaStreamDestroy(st2);
  }
  if (g->st) cudaStreamDestroy(g->st);
  delete g;
  return EDA_OK;
}

EDA_API const char* eda_group_last_error(const eda_group* g) { return g ? g->err.c_str() : eda_last_error(nullptr); }

EDA_API int eda_group_set_trajectories(eda_group* g, const double* const* xb, const double* const* y) {
  if (!g || !xb || !y) return gfail(g, EDA_ERR_INVALID, "eda_group_set_trajectories: invalid argument");
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    const int rc = eda_set_trajectory(h, xb[pi], y[pi], nullptr);
    if (rc) return gfail(g, rc, "problem " + std::to_string(pi) + ": " + h->err);
    // the group's right-hand sides: member vectors of every problem, concatenated
    if (enter(g)) return EDA_ERR_CUDA;
    const long long off = g->item_off[std::lower_bound(g->item_prob.begin(), g->item_prob.end(), pi) -
                                      g->item_prob.begin()];
    GCU(g, cudaMemcpyAsync(g->b + off, h->b, (size_t)h->M * h->n * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  }
  GCU(g, cudaStreamSynchronize(g->st));
  return leave(g);
}

EDA_API int eda_group_sketch(eda_group* g) {
  if (!g) return gfail(nullptr, EDA_ERR_INVALID, "group is NULL");
  if (enter(g)) return EDA_ERR_CUDA;
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    if (!h->have_traj) return gfail(g, EDA_ERR_STATE, "eda_group_sketch before eda_group_set_trajectories");
    if (h->ell < 1) continue;
    eda::count_launch();
    g_gamma_kernel<<<eda::grid_for((long long)h->ell * h->n), 256, 0, g->st>>>(h->n, h->ell, h->b, g->Phi + g->sk_off[pi]);
    GCU(g, cudaGetLastError());
  }
  const bool fp64 = g->prec == EDA_FP64;
  int rc = set_items(g, fp64, true);
  if (rc) return rc;
  rc = group_sweep(g, fp64, g->Phi, g->Y, 0, true);
  if (rc) return rc;
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    if (h->ell < 1) continue;
    const size_t bytes = (size_t)h->ell * h->n * sizeof(double);
    GCU(g, cudaMemcpyAsync(h->Phi, g->Phi + g->sk_off[pi], bytes, cudaMemcpyDeviceToDevice, g->st));
    GCU(g, cudaMemcpyAsync(h->Y, g->Y + g->sk_off[pi], bytes, cudaMemcpyDeviceToDevice, g->st));
    h->have_sketch = true;
    h->have_lmp = false;
  }
  GCU(g, cudaStreamSynchronize(g->st));
  int rc2 = set_items(g, fp64, false);
  if (rc2) return rc2;
  if (g->prec == EDA_MIXED) rc2 = set_items(g, true, false);
  if (rc2) return rc2;
  GCU(g, cudaStreamSynchronize(g->st));
  return leave(g);
}

EDA_API int eda_group_build_lmp(eda_group* g) {
  if (!g) return gfail(nullptr, EDA_ERR_INVALID, "group is NULL");
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    if (h->ell < 1) continue;
    const int rc = eda_build_lmp(h, nullptr, nullptr);
    if (rc) return gfail(g, rc, "problem " + std::to_string(pi) + ": " + h->err);
  }
  return EDA_OK;
}

EDA_API int eda_group_autotune(eda_group* g, double* best_ms_out) {
  if (!g) return gfail(nullptr, EDA_ERR_INVALID, "group is NULL");
  if (enter(g)) return EDA_ERR_CUDA;
  for (int pi = 0; pi < g->P; ++pi)
    if (!g->hs[pi]->have_traj) return gfail(g, EDA_ERR_STATE, "eda_group_autotune before eda_group_set_trajectories");
  const bool fp64 = g->prec == EDA_FP64;
  // tile shapes (1 or 2 times the fewest CTAs per member) x halo refresh
  // periods K in {2, 4, 8, 16}: time the batched member sweep of every
  // bucket alone and charge each problem its share of the bucket's time (by
  // members x n x window); keep each problem's cheapest shape and period
  const int Ks[] = {2, 4, 8, 16};
  std::vector<int> bestK(g->P, 4), bestM(g->P, 1);
  std::vector<double> bestT(g->P, 1e300);
  std::vector<double> work(g->P);
  for (int pi = 0; pi < g->P; ++pi)
    work[pi] = (double)g->hs[pi]->M * g->hs[pi]->n * std::max(g->hs[pi]->N, 1);
  cudaEvent_t e0, e1;
  GCU(g, cudaEventCreate(&e0));
  GCU(g, cudaEventCreate(&e1));
  GCU(g, cudaMemcpyAsync(g->p, g->b, (size_t)g->vtot * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  GCU(g, cudaMemsetAsync(g->active, 0xFF, (size_t)g->T * sizeof(int), g->st));  // all flags nonzero
  double total = 0.0;
  for (int m : {1, 2})
  for (int K : Ks) {
    std::vector<int> Kp(g->P, K), Mp(g->P, m);
    int rc = plan_group(g, fp64, Kp, Mp);
    if (rc) return rc;
    rc = set_items(g, fp64, false);
    if (rc) return rc;
    std::vector<Bucket>& bs = fp64 ? g->b64 : g->b32;
    for (Bucket& b : bs) {
      if (b.items.empty()) continue;
      // time this bucket alone
      std::vector<Bucket> only(1, b);
      std::swap(bs, only);
      float ms = 0.f;
      for (int rep = -1; rep < 2; ++rep) {
        if (rep == 0) GCU(g, cudaEventRecord(e0, g->st));
        rc = group_sweep(g, fp64, g->p, g->q, 1, false);
        if (rc) return rc;
      }
      GCU(g, cudaEventRecord(e1, g->st));
      GCU(g, cudaEventSynchronize(e1));
      GCU(g, cudaEventElapsedTime(&ms, e0, e1));
      std::swap(bs, only);
      double bw = 0.0;
      for (int pi : b.probs) bw += work[pi];
      for (int pi : b.probs) {
        const double cost = (double)ms * work[pi] / std::max(bw, 1.0);
        if (cost < bestT[pi]) {
          bestT[pi] = cost;
          bestK[pi] = K;
          bestM[pi] = m;
        }
      }
    }
  }
  int rc = plan_group(g, fp64, bestK, bestM);
  if (rc) return rc;
  rc = set_items(g, fp64, false);
  if (rc) return rc;
  // time the tuned batched sweep of the whole group
  float ms = 0.f;
  for (int rep = -1; rep < 2; ++rep) {
    if (rep == 0) GCU(g, cudaEventRecord(e0, g->st));
    rc = group_sweep(g, fp64, g->p, g->q, 1, false);
    if (rc) return rc;
  }
  GCU(g, cudaEventRecord(e1, g->st));
  GCU(g, cudaEventSynchronize(e1));
  GCU(g, cudaEventElapsedTime(&ms, e0, e1));
  total = ms / 2.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
    g->g_key = -1;
  }
  if (eda::env_int("EDA_VERBOSE", 0)) {
    std::vector<Bucket>& bs = fp64 ? g->b64 : g->b32;
    for (const Bucket& b : bs)
      std::fprintf(stderr, "eda_group_autotune: bucket CS=%d A=%d K=%d problems=%zu items=%zu\n", b.CS, b.A, b.K,
                   b.probs.size(), b.items.size());
  }
  if (best_ms_out) *best_ms_out = total;
  return leave(g);
}

EDA_API int eda_group_solve(eda_group* g, double tol, int maxit, int use_lmp, double* const* dz_out, int* iters_out,
                            double* relres_out, int* status_out) {
  if (!g) return gfail(nullptr, EDA_ERR_INVALID, "group is NULL");
  if (maxit < 0 || !(tol >= 0.0)) return gfail(g, EDA_ERR_INVALID, "eda_group_solve: invalid argument");
  for (int pi = 0; pi < g->P; ++pi) {
    eda_handle* h = g->hs[pi];
    if (!h->have_traj) return gfail(g, EDA_ERR_STATE, "eda_group_solve before eda_group_set_trajectories");
    if (use_lmp && h->k > 0 && !h->have_lmp) return gfail(g, EDA_ERR_STATE, "eda_group_solve before the LMPs");
  }
  const bool mixed = g->prec == EDA_MIXED;
  if (enter(g)) return EDA_ERR_CUDA;
  GCU(g, cudaMemsetAsync(g->nactive, 0, sizeof(int), g->st));
  GCU(g, cudaMemsetAsync(g->x, 0, (size_t)g->vtot * sizeof(double), g->st));
  GCU(g, cudaMemcpyAsync(g->r, g->b, (size_t)g->vtot * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  GCU(g, eda::pcg_start<double>(0, g->T, g->b, g->r, g->sc, g->active, tol, g->nactive, g->st, g->d_n_of,
                                g->d_off_of));
  const char* taus = std::getenv("EDA_MIXED_INNER_TOL");
  const double tau = (taus && *taus) ? std::atof(taus) : 1e-3;
  if (mixed && tol > 0.0 && tau > 0.0) {
    eda::count_launch();
    g_set_tolm_kernel<<<eda::grid_for(g->T), 256, 0, g->st>>>(g->T, g->sc, tol, tau);
    GCU(g, cudaGetLastError());
  }
  int it = 0;
  int rc = group_pcg_loop(g, !mixed, use_lmp != 0, tol, maxit, &it);
  if (rc) return rc;
  if (mixed) {
    for (int rep = 0; rep < 64; ++rep) {
      // FP64 true residual of every member (FP64 group sweep on x)
      GCU(g, cudaMemsetAsync(g->active, 0xFF, (size_t)g->T * sizeof(int), g->st));
      rc = group_sweep(g, true, g->x, g->q, 1, false);
      if (rc) return rc;
      GCU(g, cudaMemsetAsync(g->dflag, 0, sizeof(int), g->st));
      // members not reactivated below stay inactive
      GCU(g, cudaMemsetAsync(g->active, 0, (size_t)g->T * sizeof(int), g->st));
      eda::count_launch();
      g_true_res_kernel<<<g->T, 256, 0, g->st>>>(g->d_n_of, g->d_off_of, g->b, g->q, g->r, g->sc, g->active,
                                                 tol > 0.0 ? tol : 1e300, g->nactive, g->dflag, tau > 0.0 ? tau : 0.0,
                                                 maxit);
      GCU(g, cudaGetLastError());
      int need = 0;
      GCU(g, cudaMemcpyAsync(g->hring, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->st));
      GCU(g, cudaStreamSynchronize(g->st));
      need = g->hring[0];
      if (need == 0 || tol <= 0.0) break;
      rc = group_pcg_loop(g, false, use_lmp != 0, tol, maxit, &it);
      if (rc) return rc;
    }
  }
  // outputs
  if (dz_out) {
    for (int pi = 0; pi < g->P; ++pi) {
      if (!dz_out[pi]) continue;
      eda_handle* h = g->hs[pi];
      const long long off = g->item_off[std::lower_bound(g->item_prob.begin(), g->item_prob.end(), pi) -
                                        g->item_prob.begin()];
      GCU(g, cudaMemcpyAsync(dz_out[pi], g->x + off, (size_t)h->M * h->n * sizeof(double), cudaMemcpyDefault, g->st));
    }
  }
  int* dit = nullptr;
  double* drr = nullptr;
  int* dst = nullptr;
  const int T = g->T;
  GCU(g, cudaMallocAsync((void**)&dit, T * sizeof(int), g->st));
  GCU(g, cudaMallocAsync((void**)&drr, T * sizeof(double), g->st));
  GCU(g, cudaMallocAsync((void**)&dst, T * sizeof(int), g->st));
  eda::count_launch();
  g_export_kernel<<<eda::grid_for(T), 256, 0, g->st>>>(T, g->sc, dit, drr, dst);
  GCU(g, cudaGetLastError());
  if (iters_out) GCU(g, cudaMemcpyAsync(iters_out, dit, T * sizeof(int), cudaMemcpyDefault, g->st));
  if (relres_out) GCU(g, cudaMemcpyAsync(relres_out, drr, T * sizeof(double), cudaMemcpyDefault, g->st));
  if (status_out) GCU(g, cudaMemcpyAsync(status_out, dst, T * sizeof(int), cudaMemcpyDefault, g->st));
  GCU(g, cudaFreeAsync(dit, g->st));
  GCU(g, cudaFreeAsync(drr, g->st));
  GCU(g, cudaFreeAsync(dst, g->st));
  GCU(g, cudaStreamSynchronize(g->st));
  return leave(g);
}

}  // extern "C"
