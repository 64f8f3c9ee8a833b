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
// (x ~ hi + lo), each product taken as hi.hi + hi.lo + lo.hi.  tiles: the
// lmp_tc_elems(n, k) BF16 copies of S that split_bf16 writes.  W scratch
// [Mp x kt] FP32 with kt = lmp_tc_kt(k) and Mp = M rounded up to 16 (zeroed
// here).  *timeout (device int) is set when a bounded wait (for the bulk
// copies or the tensor core) gives up (that CTA then skips its outputs).
// k <= 128; any M (tiles of at most 256 members).
cudaError_t lmp_apply_tc(int n, int k, const __nv_bfloat16* tiles, const double* coef, int M, const double* R,
                         double* Z, const int* active, float* W, int* timeout, cudaStream_t s);

// The padded sizes: k rounded up to 16, n to whole chunks of 128 rows.
int lmp_tc_kt(int k);
int lmp_tc_ns(int n);
// BF16 elements of the tiled copies of S: per chunk of 128 rows, the
// projection operand (128 modes x 128 rows) and the expansion operand (128
// rows x kt modes), each as high and low parts, in the core-matrix layout
// of the MMA's shared-memory operands.
size_t lmp_tc_elems(int n, int k);

// Writes the tiled copies of S [k x n] (FP64, column-major) into tiles:
// hi = bf16(s), lo = bf16(s - hi), zero outside k x n.
cudaError_t split_bf16(int n, int k, const double* S, __nv_bfloat16* tiles, cudaStream_t s);

}  // namespace eda
