// Batched application of the spectral LMP and of its symmetric factor
// (Section 3.1): Z[m] = R[m] + S diag(coef) S^T R[m] for every active member
// m, S the k orthonormal columns (k x n column-major), coef the k
// coefficients (theta / (1 + lambda_i) - 1 for P_theta, sqrt(theta) /
// sqrt(1 + lambda_i) - 1 for U_theta).  Two launches: the projections
// W = S^T R (row chunks, atomics into W), then the expansion
// Z = R + S (coef o W).  Z may alias R.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace eda {

// CUDA cores, LMP arithmetic in TS (double: FP64; float: FP32 with the FP32
// copy of S); W scratch [M][kpad] of TS with kpad >= k (zeroed here).
template <typename TS>
cudaError_t lmp_apply_cc(int n, int k, const TS* S, const double* coef, int M, const double* R, double* Z,
                         const int* active, TS* W, int kpad, cudaStream_t s);

// Tensor cores (tcgen05, kind::f16 with BF16 operands, FP32 accumulation in
// tensor memory): S and each R split into BF16 high and low parts
// (x ~ hi + lo), each product taken as hi.hi + hi.lo + lo.hi.  Shi / Slo:
// [kt x nS] and ShiT / SloT: [nS x kt] BF16 copies of S from split_bf16
// (kt = lmp_tc_kt(k), nS = lmp_tc_ns(n), zero padding).  W scratch
// [Mp x kt] FP32 with Mp = M rounded up to 16 (zeroed here).  *timeout
// (device int) is set when a bounded wait on the tensor core gives up (that
// CTA then skips its outputs).  k <= 128; any M (groups of 256 members).
cudaError_t lmp_apply_tc(int n, int k, const __nv_bfloat16* Shi, const __nv_bfloat16* Slo,
                         const __nv_bfloat16* ShiT, const __nv_bfloat16* SloT, const double* coef, int M,
                         const double* R, double* Z, const int* active, float* W, int* timeout, cudaStream_t s);

// The padded sizes of the BF16 copies: k rounded up to 16, n to 128.
int lmp_tc_kt(int k);
int lmp_tc_ns(int n);

// The four BF16 copies of S [k x n] (FP64, column-major): hi = bf16(s),
// lo = bf16(s - hi), zero outside k x n.
cudaError_t split_bf16(int n, int k, const double* S, __nv_bfloat16* Shi, __nv_bfloat16* Slo, __nv_bfloat16* ShiT,
                       __nv_bfloat16* SloT, cudaStream_t s);

}  // namespace eda
