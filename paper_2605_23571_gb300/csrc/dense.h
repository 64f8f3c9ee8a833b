// Launchers of the dense kernels (dense.cu).
#pragma once

#include <cuda_runtime.h>

#include "../../include/eda.h"
#include "eda_internal.h"

namespace eda {

// Per-member CG scalars (FP64 recurrences, Section 2.3).
struct PcgScalars {
  double rz;      // (unused: r . z lives in the iteration accumulators)
  double bnorm;   // ||b||
  double relres;  // ||r|| / ||b||
  int iters;
  int status;
  double tolm;    // per-member inner threshold of a refinement round on ||r||/||b|| (0: none)
  double errb;    // certified relative-error bound ||r|| / (||x|| - ||r||) of the last
                  // FP64 true residual (NaN until one is taken)
};

template <typename TA, typename TB>
cudaError_t gemm_tn(int n, const TA* A, int ka, const TB* B, int mb, double* Cm, int ldc,
                    const int* active_cols, bool sym, cudaStream_t s);
template <typename TA, typename TZ>
cudaError_t gemm_nn(int n, const TA* A, int k, int m, const double* Bs, const double* scale, const TZ* R,
                    TZ* Z, const int* active_cols, cudaStream_t s);
cudaError_t chol_inv(const double* G, int m, double shift, double* R, double* Rinv, int* status,
                     cudaStream_t s);
cudaError_t tri_mul(const double* A, const double* B, double* P, int m, cudaStream_t s);
cudaError_t nystrom_core(const double* W, const double* RY, int m, int k, double nu, int theta_mode,
                         double theta_given, double* UT, double* D, double* cvec, double* theta_out,
                         int* status, cudaStream_t s);
// Algorithm 1 core for a numerically rank-deficient sketch (truncated
// eigendecompositions, Appendix B), around two caller GEMMs:
// robust_winv: M [m x m] = U mu^{-1/2} over W's eigenvalues above rtol*max
// (zero columns elsewhere); the caller forms Z = Y M and K = Z^T Z;
// robust_eig: SB [m x k] = V D^{-1/2} for the first k_eff modes of K =
// V D V^T (S = Z SB), D, c, theta, *rank_out = k_eff.
cudaError_t robust_winv(const double* W, int m, double rtol, double* M, cudaStream_t s);
cudaError_t robust_eig(const double* K, int m, int k, double rtol, int theta_mode, double theta_given, double* SB,
                       double* D, double* cvec, double* theta_out, int* rank_out, cudaStream_t s);
// Start of the batched PCG, one CTA per item: ||b||, the relative residual
// of the initial r, statuses and the active set.  With n_of/off_of, item j
// has length n_of[j] at offset off_of[j]; otherwise length n at j*n.  The
// iterations are in pcg.h.
template <typename T>
cudaError_t pcg_start(int n, int m, const double* b, const T* r, PcgScalars* sc, int* active, double tol,
                      int* nactive, cudaStream_t s, const int* n_of = nullptr, const long long* off_of = nullptr);
template <typename TS, typename TD>
cudaError_t convert(long long count, const TS* src, TD* dst, cudaStream_t s);

}  // namespace eda
