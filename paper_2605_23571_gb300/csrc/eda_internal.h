// Internal declarations shared by the translation units of libeda.so.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/eda.h"

namespace eda {

// Process-wide count of kernel launches (tracing).
void count_launch(int k = 1);

enum SweepMode { MODE_HVP = 0, MODE_RHS = 1, MODE_NL = 2 };

// One problem of a group launch (uneven batching): its model, observation
// network, U_B taps, trajectory store and sweep tiling (the launch fixes the
// cluster size and the run length C; each problem has its own tile, halo,
// refresh period and number of active threads A).
template <typename T>
struct SweepProb {
  int n, N, p, w, nos;
  int Ttile, HL, E, K, A;
  T F, dt;
  const T* traj;
  long long traj_mstride;
  const int* obs_of_t;
  const int* obs_ptr;
  const int* obs_idx;
  const T* rinv;
  const int* obs_tab;
  const T* bcoef;
};

// One work item of a group launch: a vector of problem `prob` on the
// trajectory of `member`, at offset voff of the launch's concatenated
// input/output arrays and soff of its stash (observation space); flag >= 0
// indexes an activity flag (the item is skipped when it is 0).
struct SweepItem {
  int prob, member, flag, pad;
  long long voff, soff;
};

// Arguments of one launch of the Lorenz-96 sweep kernel.  One "column" is one
// vector processed on the trajectory of member col_member[col]; it is split
// over CS CTAs (a thread-block cluster), CTA r owning global indices
// [r*Ttile, min((r+1)*Ttile, n)) and computing redundantly on the extended
// region of E = A*C elements starting HL to the left of its tile.  The halo is
// refreshed from its owners every K steps.
template <typename T>
struct SweepArgs {
  int n, N;
  T F, dt;
  // trajectory store, states 0..N of each member (MODE_HVP / MODE_RHS)
  const T* traj;
  long long traj_mstride;
  // observation network
  const int* obs_of_t;   // [N+1]: observation-step index at step t, or -1
  const int* obs_tab;    // [CS][nos][8] observation ranges per CTA (or nullptr)
  int nos;
  const int* obs_ptr;    // [n_obs_times + 1]
  const int* obs_idx;    // [p]
  const T* rinv;         // [p]
  int p;
  // U_B taps
  int w;
  const T* bcoef;        // [w+1]
  // columns
  int ncol;
  const int* col_member; // [ncol] or nullptr (= column index)
  int M;                 // members in the trajectory store: a column whose
                         // col_member is outside [0, M) gets NaN outputs
                         // (0: not checked; the group launch's items are)
  const int* col_active; // [ncol] or nullptr (= all active)
  const T* V;            // MODE_HVP input vectors [ncol][v_stride]
  long long v_stride;
  T* OUT;                // MODE_HVP / MODE_RHS outputs
  long long out_stride;
  const double* V64;     // if set: FP64 input vectors instead of V (FP32 sweeps)
  double* OUT64;         // if set: FP64 outputs instead of OUT
  T* stash;              // MODE_HVP: per-column obs stash [ncol][stash_stride]
                         // MODE_RHS: per-member forcing R^{-1} d [member][stash_stride]
  long long stash_stride;
  int include_identity;
  // MODE_HVP with include_identity: if set, dot_out[item * dot_stride] +=
  // v . (H v) over the column (item = column, or the group item's flag)
  double* dot_out;
  int dot_stride;
  int mode;
  // MODE_NL
  const T* x0;           // [col][x0_stride] initial states
  long long x0_stride;
  T* traj_out;           // [member][N+1][n] or nullptr
  long long traj_out_mstride;
  T* final_out;          // [col][n] final state or nullptr
  const T* yobs;         // [col][p] or nullptr (then d = H x)
  T* d_out;              // [col][p] or nullptr
  T* rd_out;             // [col][p] or nullptr: R^{-1} d
  // Stage store of every RK4 step t -> t+1 (rows t = 0..N-1) of each
  // member: seven arrays, array s at + s * stage_astride, member m at
  // + m * traj_mstride (the trajectory's layout): 0-2 the stage states X2,
  // X3, X4; 3-6 the stencil differences D_j = X_{j+1} - X_{j-2} of X1 = x_t,
  // X2, X3, X4.  MODE_NL with stage_out writes them; MODE_HVP / MODE_RHS with
  // stages read them instead of recomputing (three FP64 instructions per
  // tangent-linear or adjoint slope instead of five).
  T* stage_out;
  const T* stages;
  long long stage_astride;
  // checkpointed trajectory (multi-launch plans only): ckpt > 0 means traj
  // holds the states x_{j ckpt} only (row j); MODE_NL stores those rows, and
  // the Hessian-product and right-hand-side launches recompute the states of
  // their K = ckpt steps from the segment's checkpoint into shared memory at
  // byte offset xseg_off
  int ckpt;
  int xseg_off;
  // plan
  int CS, Ttile, HL, E, K;
  // multi-launch mode (n too large for one cluster): CS tiles per column
  // without a cluster, this launch runs forward steps [f0, f1) and backward
  // steps b1-1 down to b0, loading the state of its extended region from
  // st_in [col][n] and storing its owned tile to st_out [col][n]
  int ml, f0, f1, b1, b0;
  const T* st_in;
  T* st_out;
  // warp-tiled plans: [CS][warps][nos][8] observation ranges of each warp
  // (injection: k0, k1, offset for two segments; gather: k0, k1)
  const int* wtab;
  // group launch (uneven batching): when items != nullptr, column c of the
  // launch is items[c] and every problem field above comes from probs[prob]
  const SweepProb<T>* probs;
  const SweepItem* items;
  const int* flags;
};

// Largest halo refresh period a tiling accepts (the halo 8K + 8 must stay
// far from int overflow; windows are much shorter).
constexpr int kMaxRefresh = 4096;

struct SweepPlan {
  int CS, C, A, E, Ttile, HL, K;
  size_t smem;
  int ml;    // 1: multi-launch tiles of K steps (no cluster), CS = tiles per column
  int warp;  // 1: warp-tiled Hessian-product kernel (MODE_HVP only; needs a warp table)
  int ckpt;  // > 0: checkpointed trajectory every ckpt = K steps (multi-launch only)
};

// Picks the tiling of a sweep for state size n (elem_bytes = sizeof(T)):
// the smallest cluster size >= min_cs whose tile fits one CTA.  K_hint > 0
// fixes the halo refresh period, C > 0 the values per thread (as in
// plan_sweep_exact).  Returns false if no plan fits.
bool plan_sweep(int n, int elem_bytes, int w, int min_cs, int K_hint, SweepPlan* out, int C = 0);

// Dynamic shared memory of a sweep launch with A threads, runs of C and
// at most w+1 taps.
size_t sweep_smem_bytes(int A, int C, int w, int elem_bytes);

// A multi-launch plan: tiles of A*C - 2HL owned points, K steps per launch,
// A threads per CTA (A = 0: 512 for FP64, 256 for FP32, 256 checkpointed;
// else a multiple of 32 up to 512).  ckpt: a checkpointed plan (K = the
// checkpoint period, halo ckpt_halo(K), K states of the region in shared
// memory).
bool plan_sweep_ml(int n, int elem_bytes, int w, int K, int A, SweepPlan* out, bool ckpt = false);

// Halo of a checkpointed multi-launch plan: a backward launch recomputes
// its K states from the checkpoint (their edge errors reach 8 points per
// step from the left end of the region and 4 from the right) and the
// adjoint spreads errors 11 points per step both ways: 8(K-1) + 11K + 1 on
// the left, rounded up to 19K + 8.
inline int ckpt_halo(int K) { return 19 * K + 8; }

// A warp-tiled Hessian-product plan with cluster size CS, refresh period K
// and C values per lane (FP64 2 or 4, FP32 4 or 8): warps of 32*C points
// owning all but a halo of 12 (C = 2, 4) or 16 (C = 8) at each end, at most
// 16 warps per CTA, and a CTA region no longer than n.  False if it does
// not fit.
bool plan_sweep_warp(int n, int elem_bytes, int w, int CS, int K, int C, SweepPlan* out);

// The observation table of a warp-tiled plan (see SweepArgs::wtab).
void warp_obs_table(const SweepPlan& p, int n, int nos, const int* obs_ptr, const int* obs_idx, int* tab);

// The plan with exactly cluster size CS, refresh period K and C values per
// thread (C = 0: 4 for FP64, 8 for FP32; else FP64 2 or 4, FP32 2, 4 or 8),
// if it fits.
bool plan_sweep_exact(int n, int elem_bytes, int w, int CS, int K, SweepPlan* out, int C = 0);

// Per-CTA observation ranges of a plan: for CTA r and observation step j,
// tab[(r*nos + j)*8 + 0..1] = [k0, k1) of the observations of the owned tile,
// [2..4] and [5..7] = (k0, k1, base) of the (at most two) index ranges of the
// extended region, local position = obs_idx[k] - base.  Empty when the
// extended region is longer than n (then the kernel scans every observation).
void obs_table(const SweepPlan& p, int n, int nos, const int* obs_ptr, const int* obs_idx,
               int* tab /* [CS*nos*8] */, bool* usable);

// Launches the sweep for `ncol` columns.  Returns a cudaError_t.  A
// multi-launch plan needs ml_buf: two state buffers of ncol * n values.
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, const SweepPlan& plan, cudaStream_t s, T* ml_buf0 = nullptr,
                         T* ml_buf1 = nullptr);

}  // namespace eda
