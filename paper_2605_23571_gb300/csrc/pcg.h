// Batched preconditioned CG (Section 2.3) with the scaled spectral LMP
// (Section 3.1), one iteration as four launches over row chunks of all
// members of all problems:
//   sweep   q = H p, with p^T q accumulated per member in its epilogue;
//   update  alpha = r.z / p.q, x += alpha p, r -= alpha q, ||r||^2 and the
//           LMP projections w = S^T r (split over row chunks);
//   precond the per-member stopping test, z = r + S diag(c) w, r.z;
//   dir     beta = (r.z)_new / (r.z)_old, p = z + beta p.
// Reductions over rows go to per-member accumulators with atomics.  r.z is
// double-buffered by iteration parity and every accumulator is zeroed by a
// launch that does not read it, so no launch reads a value that another CTA
// of the same launch writes.  The per-member stopping test is taken by every
// CTA from values no CTA of that launch writes; the CTA of a problem's first
// row chunk records it.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "dense.h"

namespace eda {

// Per-member accumulators of one iteration (56 bytes: pq is the first
// double, so the sweep epilogue adds p^T q at acc + kPcgAccStride * member).
struct PcgAcc {
  double pq;     // p^T q of this iteration (sweep epilogue)
  double rr;     // ||r||^2 after the update
  double rz[2];  // r^T z by iteration parity
  double xx;     // ||x||^2 after the update (certified error test)
  double jx;     // x^T (b + r) after the update (cost record: J = -jx / 2)
  int inc;       // 1: the member iterated (set by precond, counted by dir)
  int pad;
};
constexpr int kPcgAccStride = (int)(sizeof(PcgAcc) / sizeof(double));

// One problem of the batch: members item0 .. item0+M-1, member m's vectors
// at off0 + m * n of the concatenated layout; S is k x n column-major (TS),
// c the k LMP coefficients (k = 0: no LMP).  Solve options of the problem:
// etol > 0 adds the certified error test ||r|| / (||x|| - ||r||) <= etol to
// the stopping rule (lambda_min(I + A) >= 1, Section 2.3, makes it a bound
// on ||x - x*|| / ||x*||); jhist != nullptr records the quadratic cost
// J(x_i) = 1/2 x^T H x - b^T x = -x^T (b + r) / 2 of every iterate at
// jhist[m * jstride + i] (b: the right-hand sides, read only then).
struct PcgProb {
  int n, M, k, item0;
  long long off0;
  const void* S;
  const double* c;
  double etol;
  const double* b;
  double* jhist;
  int jstride;
};

// A chunk of rows [row0, row0 + rows) of one problem (rows <= kPcgRows);
// first = 1 for the chunk with row0 = 0, whose CTA does the problem's
// per-member bookkeeping.
struct PcgTask {
  int prob, row0, rows, first;
};
constexpr int kPcgRows = 128;

// Where the kernels find their row chunks and problems: the task and problem
// tables (device memory; the group path), or, with single != 0, the one
// problem `one` passed by value with row chunk blockIdx.x (a handle's solve:
// no table loads ahead of the work).  ntasks: row chunks of the launch.
struct PcgGrid {
  const PcgTask* tasks;
  const PcgProb* probs;
  int ntasks;
  int single;
  PcgProb one;
};

// The grid of one problem: ceil(prob.n / kPcgRows) row chunks, the problem
// by value.
PcgGrid pcg_single(const PcgProb& prob);
// The grid of the task and problem tables (ntasks row chunks).
PcgGrid pcg_tables(const PcgTask* tasks, int ntasks, const PcgProb* probs);

// Builds the row-chunk tasks of the given problem sizes.  Every kernel
// below runs a grid of (row chunks, ceil(mmax / 8)) CTAs of 8 warps, one
// member per warp (mmax: the largest member count of the problems).
void pcg_tasks(const int* n_of, int nprob, std::vector<PcgTask>* out);

// Zeroes the accumulators of every member and its projections (start of a
// PCG loop).
cudaError_t pcg2_reset(PcgAcc* acc, int T, void* Wk, size_t wk_bytes, cudaStream_t s);

// update = 1: the CG update and the projections of the new r.
// update = 0: projections of the current r only (start of a loop).
// use_lmp = 0: no projections.
template <typename TS>
cudaError_t pcg2_update(const PcgGrid& G, int kmax, int mmax, const double* p,
                        const double* q, double* x, double* r, PcgScalars* sc, PcgAcc* acc, int* active, TS* Wk,
                        int par, int update, int use_lmp, int* nactive, cudaStream_t s);

// init = 0: stopping test (tol, maxit, fixed), then z and r.z into slot
// par^1 for the members that go on.  init = 1 (start of a loop): no test;
// z, p = z and r.z into slot 0; the caller then clears the projections
// before the first update.
// zpre != nullptr: z = P r was computed by a separate LMP launch (the
// tensor-core LMP) and is read from zpre instead (use_lmp must be 0).
template <typename TS>
cudaError_t pcg2_precond(const PcgGrid& G, int kmax, int mmax, const double* r,
                         double* z, double* p, PcgScalars* sc, PcgAcc* acc, int* active, const TS* Wk, int par,
                         double tol, int maxit, int fixed, int use_lmp, int init, int* nactive, cudaStream_t s,
                         const double* zpre = nullptr);

// p = z + beta p; counts the iteration and clears rr and the projections.
// With host_count (pinned host memory) != NULL, one thread also copies the
// active count *nactive there, which the host reads after an event.
template <typename TS>
cudaError_t pcg2_dir(const PcgGrid& G, int kmax, int mmax, const double* z, double* p,
                     PcgScalars* sc, PcgAcc* acc, const int* active, TS* Wk, int par, cudaStream_t s,
                     const int* nactive = nullptr, int* host_count = nullptr);

// Residual replacement: r = b - hx (hx = (I + A) x from an accurate sweep)
// and ||r||^2 (cleared first) for the active members of T.
cudaError_t pcg2_replace(const PcgGrid& G, int mmax, const double* b,
                         const double* hx, double* r, PcgAcc* acc, int T, const int* active, cudaStream_t s);

// acc[col].pq += v_col . hv_col for active columns of an [ncol][n] batch
// (used where the sweep epilogue cannot accumulate it).
cudaError_t pcg2_col_dot(int n, int ncol, const double* v, const double* hv, const int* active, PcgAcc* acc,
                         cudaStream_t s);

// ------------------------------------------------------------------------
// Persistent PCG (one launch per solve phase): one thread-block cluster per
// member runs the whole iteration -- the sweep q = (I + A) p of its column,
// then alpha, x, r, ||r||^2, ||x||^2 and the LMP projections S^T r on each
// CTA's tile, the stopping test, z = r + S (c o w), r.z, beta and p -- with
// the reductions through per-member global accumulators (atomics, then a
// cluster barrier) and no host involvement, until the member stops.

// Accumulators of one member, by iteration parity (a slot is cleared one
// iteration after it was read; zeroed before the launch).
struct PersistAcc {
  double pq[2], rr[2], xx[2], rz[2];
  double ex[2];  // the launch's exit flag as rank 0 read it (1: leave at this iteration's end)
};

template <typename T>
struct PersistArgs {
  SweepArgs<T> sw;      // MODE_HVP of column m on member m: V = p, OUT = q, identity included
  int n, M, k, kmax;
  double *x, *r, *z, *p, *q;  // [M][n]
  const T* S;           // k x n column-major, the LMP arithmetic type
  const double* c;      // k coefficients
  PcgScalars* sc;
  PcgAcc* acc;          // r.z of the loop start (slot 0, from pcg2_precond with init,
                        // or saved there by a launch that left early)
  int* active;
  int* nactive;
  double tol, etol;
  int maxit, fixed, use_lmp;
  PersistAcc* pacc;     // [M]
  T* W;                 // [2][M][kmax] projections by parity
  // early exit (re-tiling of the convergence tail): when a member's stop
  // leaves at most exit_below members active, the stopping cluster sets
  // *brk, and every other cluster leaves at the end of its current
  // iteration with its PCG state saved (x, r, z, p in place; r.z in
  // acc[j].rz[0], the iteration count and residual in sc[j]; still active)
  // for a launch with another tiling.  brk == nullptr: no early exit.
  int exit_below;
  int* brk;
  // group mode (items != nullptr): the clusters take the launch's items
  // (one member of one problem each, largest problems first) from a
  // device-side queue; item i is sw.items[i], its PCG index (into sc, acc,
  // active, pacc and W, with M the group's total) is items[i].flag, its
  // problem's vector layout and LMP pprobs[items[i].prob]
  const SweepItem* items;
  int nitems;
  const PcgProb* pprobs;
  int* queue;           // next item to take (zeroed before the launch)
};

// Launches the persistent PCG over the M members (a cluster tiling, not
// multi-launch, not warp-tiled).  In group mode, plan describes the bucket
// (cluster size, threads, run length, shared memory) and the grid holds as
// many clusters as fit on the device at once.  With query != nullptr nothing
// is launched: *query receives how many of the launch's clusters fit on the
// device at once (0: the plan cannot run).  Returns a cudaError_t.
template <typename T>
cudaError_t launch_pcg_persist(const PersistArgs<T>& a, const SweepPlan& plan, cudaStream_t s,
                               int* query = nullptr);

}  // namespace eda
