// The EDA handle and the internal helpers shared by api.cu and group.cu.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dense.h"
#include "eda_internal.h"
#include "pcg.h"

using eda::PcgScalars;
using eda::SweepArgs;
using eda::SweepPlan;

struct eda_handle {
  // problem
  int n = 0, N = 0, M = 0, p = 0, nos = 0, w = 0, ell = 0, k = 0;
  int theta_mode = 0, precision = 0, ckpt = 0;
  int trows = 0;  // rows of each member's trajectory store (N + 1, or N / ckpt + 1 checkpoints)
  double F = 8.0, dt = 0.025, theta_given = 1.0;
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<int> h_obs_of_t;
  // device: problem definition
  int* obs_of_t = nullptr;
  int* obs_ptr = nullptr;
  int* obs_idx = nullptr;
  double* rinv = nullptr;
  float* rinv32 = nullptr;
  double* bcoef = nullptr;
  float* bcoef32 = nullptr;
  // device: setup products
  double* traj = nullptr;
  float* traj32 = nullptr;
  // stage store of every RK4 step ([7][member][t][n], the trajectory's
  // layout: the stage states X2, X3, X4 and the stencil differences of X1..X4),
  // written with the trajectory and read by the FP64 sweeps; nullptr:
  // recomputed
  double* stg = nullptr;
  double* d = nullptr;
  double* rd = nullptr;
  double* b = nullptr;
  // device: sketch and LMP
  double* Phi = nullptr;
  double* Y = nullptr;
  float* V32a = nullptr;  // ell x n scratch (FP32 sweeps)
  float* V32b = nullptr;
  double* Q1 = nullptr;
  double* Q = nullptr;
  double* G = nullptr;
  double* R1 = nullptr;
  double* R1i = nullptr;
  double* R2 = nullptr;
  double* R2i = nullptr;
  double* RY = nullptr;
  double* W = nullptr;
  double* UT = nullptr;
  double* Dv = nullptr;
  double* cv = nullptr;
  double* theta = nullptr;
  int* dstatus = nullptr;
  double* S = nullptr;
  float* S32 = nullptr;
  double* lmpW = nullptr;  // k x M
  // device: PCG
  double *x = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr;
  PcgScalars* sc = nullptr;
  eda::PcgAcc* acc = nullptr;      // per-member accumulators of an iteration
  double* Wk = nullptr;            // M x max(k,1) LMP projections (FP64, or FP32 in the mixed solve)
  eda::PcgGrid pgrid{};            // the handle as a one-problem batch (by value)
  int* active = nullptr;
  int* nactive = nullptr;
  int* cols = nullptr;  // identity member map 0..max(M, ell)-1
  int* zeros = nullptr; // member map of zeros (control trajectory)
  int* hflag = nullptr; // pinned host int
  static constexpr int kRing = 4;     // iterations the host may run ahead
  int* hring = nullptr;               // pinned host copies of the active count
  cudaEvent_t ring_ev[kRing] = {};
  // stash
  double* stash = nullptr;
  float* stash32 = nullptr;
  int stash_cols = 0;
  // state
  bool have_traj = false, have_sketch = false, have_lmp = false;
  // state buffers of multi-launch sweeps (n too large for one cluster)
  double* ml64[2] = {nullptr, nullptr};
  float* ml32[2] = {nullptr, nullptr};
  long long ml64_cap = 0, ml32_cap = 0;
  double shift_used = 0.0;
  int nystrom_path = 0;  // 0 Cholesky, 1 Appendix B shift, 2 truncated eigendecomposition
  int lmp_rank = 0;      // informative LMP modes (k, or k_eff on path 2)
  // the LMP applied outside the fused PCG kernels (eda_lmp_apply, the split
  // preconditioner, the tensor-core LMP): coefficients of U_theta and
  // U_theta^{-1} [2k], the BF16 copies of S (hi, lo, and transposed), FP32 /
  // TS projection scratch, the tensor-core wait flag; versions follow the LMP
  int lmp_version = 0, uv_version = -1, bf_version = -1;
  double* uv = nullptr;
  void* Sbf = nullptr;          // tiled BF16 copies of S (lmp.h: lmp_tc_elems)
  float* Wtc = nullptr;
  long long wtc_cap = 0;        // floats
  void* Wcc = nullptr;
  long long wcc_cap = 0;        // bytes
  int* tc_timeout = nullptr;
  eda::PersistAcc* pacc = nullptr;  // persistent PCG: per-member accumulators
  void* Wp = nullptr;               // persistent PCG: projections [2][M][kmax] (FP64 or FP32)
  double* bh = nullptr;         // split PCG: U b
  double* tbuf = nullptr;       // split PCG: U p
  SweepPlan plan64{}, plan32{};
  // warp-tiled plans of the Hessian-product sweeps (warp = 0: none; the
  // plans above serve then) and their observation tables
  SweepPlan wplan64{}, wplan32{};
  int* wtab64 = nullptr;
  int* wtab32 = nullptr;
  int* tab64 = nullptr;  // per-CTA observation ranges of plan64 / plan32
  int* tab32 = nullptr;
  bool tab64_ok = false, tab32_ok = false;
  // tilings of the persistent PCG's convergence tail (eda_autotune): while at
  // most `level` members are active, the solve relaunches on `plan`, which
  // spreads each remaining member over more CTAs; levels decrease along the
  // vector ([0] FP64 sweeps, [1] FP32); empty: one launch on plan64/plan32
  struct TailPlan {
    int level = 0;
    SweepPlan plan{};
    int* tab = nullptr;  // its observation table (nullptr: none fits)
  };
  std::vector<TailPlan> tail[2];
  int* brk = nullptr;  // persistent PCG early-exit flag
  std::vector<int> h_obs_ptr, h_obs_idx;
  std::vector<void*> allocs;
  // tracing of the Hessian-product sweeps ([0] FP64 sweeps, [1] FP32):
  // event pairs around each sweep on the handle's stream, drained into the
  // totals when the pool is full or on read; column counts on the device
  bool trace_on = false;
  int trace_every = 1;     // trace one sweep in trace_every
  long long trace_seen = 0;
  std::vector<cudaEvent_t> trace_ev;      // 2 per pair
  std::vector<int> trace_kind;            // precision index per pair
  int trace_used = 0;
  double trace_ms[2] = {0.0, 0.0};
  long long trace_calls[2] = {0, 0};
  unsigned long long* trace_cols = nullptr;  // device [2]
};


namespace eda {

// Records msg as the last error (of h, and of the thread) and returns code.
int fail(eda_handle* h, int code, const std::string& msg);
// True if ptr is device (or managed) memory.
bool is_device_ptr(const void* ptr);
// Installs a sweep tiling of the handle and its observation table.
int set_plan(eda_handle* h, bool fp64, const SweepPlan& pl);
// Installs (pl != nullptr) or removes the warp-tiled Hessian-product plan.
int set_warp_plan(eda_handle* h, bool fp64, const SweepPlan* pl);
// The plan of the Hessian-product sweeps of one precision and its tables:
// the warp-tiled plan if installed, else the general plan.
const SweepPlan& hvp_plan(const eda_handle* h, bool fp64, const int** obs_tab, const int** wtab);
// State buffers for a multi-launch sweep of ncol columns (no-op for
// cluster plans); grows the handle's buffers when needed.
int ensure_ml(eda_handle* h, int ncol, bool fp64);
// Reads one device int (synchronises the stream).
int read_flag(eda_handle* h, const int* dflag, int* out);
// Integer environment variable (tiling overrides, diagnostics).
int env_int(const char* name, int dflt);
// 1D grid size for a grid-stride loop over count elements.
unsigned grid_for(long long count);

}  // namespace eda

#define CU(h, ...)                                                                               \
  do {                                                                                           \
    cudaError_t e__ = (__VA_ARGS__);                                                             \
    if (e__ != cudaSuccess) {                                                                    \
      return eda::fail((h), EDA_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__)); \
    }                                                                                            \
  } while (0)
