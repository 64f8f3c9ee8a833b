// Dense pieces of the path: tall-skinny products for the sketch
// orthogonalisation and the LMP, the small FP64 factorisations of
// Algorithm 1 (Section 3.2.3), and the per-member PCG vector updates
// (Section 2.3).  All column blocks are column-major with leading dimension n.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "dense.h"

namespace eda {
namespace {

template <typename T>
__device__ __forceinline__ double block_sum(double v, double* red) {
  // warp shuffle, then across warps through shared memory
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  return red[0];
}

// C[i + j*ldc] = sum_g A[g + i*n] * B[g + j*n]  (FP64 accumulation);
// one block per (i, j); inactive columns j (mask) are skipped.
template <typename TA, typename TB>
__global__ void gemm_tn_kernel(int n, const TA* A, int ka, const TB* B, int mb, double* Cm, int ldc,
                               const int* active_cols, int sym) {
  __shared__ double red[32];
  const int i = blockIdx.x, j = blockIdx.y;
  if (active_cols && !active_cols[j]) return;
  if (sym && i > j) return;
  const TA* a = A + (long long)i * n;
  const TB* b = B + (long long)j * n;
  double s = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) s += (double)a[g] * (double)b[g];
  s = block_sum<double>(s, red);
  if (threadIdx.x == 0) {
    Cm[i + (long long)j * ldc] = s;
    if (sym && i != j) Cm[j + (long long)i * ldc] = s;
  }
}

// Z[g + j*n] = (R ? R[g + j*n] : 0) + sum_{i<k} A[g + i*n] * Bs[i + j*k]
// (Bs is k x m column-major, FP64, optionally scaled row-wise by scale[i]).
template <typename TA, typename TZ>
__global__ void gemm_nn_kernel(int n, const TA* A, int k, const double* Bs, const double* scale,
                               const TZ* R, TZ* Z, const int* active_cols) {
  extern __shared__ double bcol[];
  const int j = blockIdx.y;
  if (active_cols && !active_cols[j]) return;
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    bcol[i] = Bs[i + (long long)j * k] * (scale ? scale[i] : 1.0);
  __syncthreads();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  double acc = R ? (double)R[g + (long long)j * n] : 0.0;
  for (int i = 0; i < k; ++i) acc += (double)A[g + (long long)i * n] * bcol[i];
  Z[g + (long long)j * n] = (TZ)acc;
}

// ---------------------------------------------------------------------------
// Small dense factorisations in one CTA (FP64).  M is m x m column-major in
// shared memory.
// ---------------------------------------------------------------------------

// In-place upper Cholesky W = C^T C; returns false on a non-positive pivot.
__device__ bool chol_upper(double* M, int m, int* flag) {
  // M[i + j*m]; result C in the upper triangle, lower set to 0
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      double d = M[j + j * m];
      for (int i = 0; i < j; ++i) d -= M[i + j * m] * M[i + j * m];
      if (!(d > 0.0) || !isfinite(d)) {
        *flag = 1;
        d = 1.0;
      }
      M[j + j * m] = sqrt(d);
    }
    __syncthreads();
    const double piv = M[j + j * m];
    for (int c = j + 1 + threadIdx.x; c < m; c += blockDim.x) {
      double s = M[j + c * m];
      for (int i = 0; i < j; ++i) s -= M[i + j * m] * M[i + c * m];
      M[j + c * m] = s / piv;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    if (i > j) M[idx] = 0.0;
  }
  __syncthreads();
  return *flag == 0;
}

// X = U^{-1} for upper-triangular U (both m x m); one thread per column.
__device__ void tri_inv_upper(const double* U, double* X, int m) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    for (int i = m - 1; i >= 0; --i) {
      double s = (i == j) ? 1.0 : 0.0;
      if (i > j) {
        X[i + j * m] = 0.0;
        continue;
      }
      for (int kk = i + 1; kk <= j; ++kk) s -= U[i + kk * m] * X[kk + j * m];
      X[i + j * m] = s / U[i + i * m];
    }
  }
  __syncthreads();
}

// P = A * B for upper-triangular A, B (m x m), P upper triangular.
__device__ void tri_mul_upper(const double* Am, const double* Bm, double* P, int m) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    double s = 0.0;
    for (int kk = i; kk <= j; ++kk) s += Am[i + kk * m] * Bm[kk + j * m];
    P[idx] = (i <= j) ? s : 0.0;
  }
  __syncthreads();
}

// G (m x m) -> Cholesky factor R (G = R^T R) and Rinv; status 1 on failure.
__global__ void chol_inv_kernel(const double* G, int m, double shift, double* R, double* Rinv,
                                int* status) {
  extern __shared__ double sm[];
  double* M = sm;
  double* X = sm + m * m;
  __shared__ int flag;
  if (threadIdx.x == 0) flag = 0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    M[idx] = 0.5 * (G[idx] + G[j + i * m]) + ((i == j) ? shift : 0.0);
  }
  __syncthreads();
  chol_upper(M, m, &flag);
  if (flag) {
    if (threadIdx.x == 0) *status = 1;
    return;
  }
  tri_inv_upper(M, X, m);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    R[idx] = M[idx];
    Rinv[idx] = X[idx];
  }
}

// RY = R2 * R1 (upper triangular products).
__global__ void tri_mul_kernel(const double* A, const double* B, double* P, int m) {
  extern __shared__ double sm[];
  double* As = sm;
  double* Bs = sm + m * m;
  double* Ps = sm + 2 * m * m;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    As[idx] = A[idx];
    Bs[idx] = B[idx];
  }
  __syncthreads();
  tri_mul_upper(As, Bs, Ps, m);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) P[idx] = Ps[idx];
}

// One-sided Jacobi SVD of T (m x m) in shared memory: on return the columns
// of T are u_i sigma_i.  Parallel round-robin pairing, one warp per pair.
__device__ void jacobi_columns(double* T, int m, int* rotated, int max_sweeps) {
  const int mp = (m + 1) & ~1;  // even count (a dummy index when m is odd)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const double tol = 1e-15;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *rotated = 0;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      for (int pr = wid; pr < mp / 2; pr += nw) {
        // round-robin pairing: index 0 fixed, the rest rotate
        int pa, pb;
        {
          auto slot = [&](int s) { return s == 0 ? 0 : 1 + (s - 1 + round) % (mp - 1); };
          pa = slot(pr);
          pb = slot(mp - 1 - pr);
        }
        if (pa >= m || pb >= m) continue;
        const int p = min(pa, pb), q = max(pa, pb);
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < m; i += 32) {
          const double tp = T[i + p * m], tq = T[i + q * m];
          al += tp * tp;
          be += tq * tq;
          ga += tp * tq;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (fabs(ga) > tol * sqrt(al * be) && ga != 0.0) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt);
          const double sn = cs * tt;
          for (int i = lane; i < m; i += 32) {
            const double tp = T[i + p * m], tq = T[i + q * m];
            T[i + p * m] = cs * tp - sn * tq;
            T[i + q * m] = sn * tp + cs * tq;
          }
          if (lane == 0) *rotated = 1;
        }
      }
      __syncthreads();
    }
    if (*rotated == 0) break;
    __syncthreads();
  }
}

// Steps of Algorithm 1 after the sketch products, in one CTA:
//   W = sym(Phi^T Y) = C^T C,  T = R_Y C^{-1},  SVD T = U_T Sigma V^T,
//   D = Sigma^2 - nu (descending), keep k; LMP coefficients.
// Outputs: UT (m x k, column-major), D (k), cvec (k), theta (1); status 1 if
// the Cholesky factorisation of W fails.
__global__ void nystrom_core_kernel(const double* W, const double* RY, int m, int k, double nu,
                                    int theta_mode, double theta_given, double* UT, double* D,
                                    double* cvec, double* theta_out, int* status) {
  extern __shared__ double sm[];
  double* M = sm;              // W -> C
  double* X = sm + m * m;      // C^{-1}
  double* T = sm + 2 * m * m;  // R_Y -> T
  double* sig = sm + 3 * m * m;
  int* order = reinterpret_cast<int*>(sig + m);
  __shared__ int flag, rotated;
  if (threadIdx.x == 0) flag = 0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    M[idx] = 0.5 * (W[idx] + W[j + i * m]);
  }
  __syncthreads();
  chol_upper(M, m, &flag);
  if (flag) {
    if (threadIdx.x == 0) *status = 1;
    return;
  }
  tri_inv_upper(M, X, m);
  // T = R_Y C^{-1}: both upper triangular
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) M[idx] = RY[idx];
  __syncthreads();
  tri_mul_upper(M, X, T, m);
  jacobi_columns(T, m, &rotated, 60);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += T[i + j * m] * T[i + j * m];
    sig[j] = sqrt(s);
  }
  __syncthreads();
  // rank of each column by descending singular value (ties by index)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < m; ++i) r += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    order[r] = j;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
    const int i = idx % m, r = idx / m;
    const int j = order[r];
    const double s = sig[j];
    UT[i + (long long)r * m] = (s > 0.0) ? T[i + j * m] / s : ((i == r) ? 1.0 : 0.0);
  }
  if (threadIdx.x == 0) {
    double lamk = 0.0;
    for (int r = 0; r < k; ++r) {
      const double s = sig[order[r]];
      double d = s * s - nu;
      if (d < 0.0) d = 0.0;
      D[r] = d;
      if (r == k - 1) lamk = 1.0 + d;
    }
    double th = theta_given;
    if (theta_mode == EDA_THETA_LAMBDA_K) th = lamk;
    if (theta_mode == EDA_THETA_MID) th = 0.5 * (lamk + 1.0);
    *theta_out = th;
    for (int r = 0; r < k; ++r) cvec[r] = th / (1.0 + D[r]) - 1.0;
    *status = 0;
  }
}

// Eigendecomposition of a symmetric PSD m x m matrix held in M (one-sided
// Jacobi: columns of M V become v_i mu_i); on return M's columns are the
// unit eigenvectors scaled by f(mu_i) and mu[] the eigenvalues, where
// f(mu) = mu^{pw} if mu > rtol * max(mu) else 0.
__device__ void psd_eig_scaled(double* M, int m, double* mu, double pw, double rtol, int* rotated) {
  jacobi_columns(M, m, rotated, 60);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += M[i + j * m] * M[i + j * m];
    mu[j] = sqrt(s);
  }
  __syncthreads();
  double mx = 0.0;
  for (int j = 0; j < m; ++j) mx = fmax(mx, mu[j]);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int j = idx / m;
    const double u = mu[j];
    const double f = (u > rtol * mx && u > 0.0) ? pow(u, pw) / u : 0.0;  // unit vector times u^pw
    M[idx] *= f;
  }
  __syncthreads();
}

// Robust core of Algorithm 1 for a numerically rank-deficient sketch
// (Appendix B, truncated eigendecomposition), in two one-CTA steps around
// two tall-skinny GEMMs done by the caller:
//   (1) W = U mu U^T (symmetrised W = Phi^T Y); M = U mu^{-1/2} over the
//       eigenvalues mu > rtol * max(mu), zero columns elsewhere, so that
//       A_N = Y W^+ Y^T = Z Z^T with Z = Y M;
//   (2) K = Z^T Z = V D V^T; the eigenvectors of A_N are S = Z V D^{-1/2}
//       and its eigenvalues D.  Only modes with D > rtol * max(D) carry
//       information, so k_eff = min(k, their count); SB (m x k) = V D^{-1/2}
//       for the first k_eff modes (descending D) and zero beyond, D and c
//       zero beyond k_eff, theta taken at mode k_eff (lambda = 1 if k_eff =
//       0); *rank_out = k_eff.
// Working from Z rather than from the Gram matrix Y^T Y keeps the small
// modes: Y^T Y squares the condition number of Y and loses every singular
// value below sqrt(eps) of the largest.
__global__ void robust_winv_kernel(const double* W, int m, double rtol, double* M) {
  extern __shared__ double sm[];
  double* Ms = sm;           // m x m
  double* mu = sm + m * m;   // m
  __shared__ int rotated;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    Ms[idx] = 0.5 * (W[idx] + W[j + i * m]);
  }
  __syncthreads();
  psd_eig_scaled(Ms, m, mu, -0.5, rtol, &rotated);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) M[idx] = Ms[idx];
}

__global__ void robust_eig_kernel(const double* K, int m, int k, double rtol, int theta_mode, double theta_given,
                                  double* SB, double* D, double* cvec, double* theta_out, int* rank_out) {
  extern __shared__ double sm[];
  double* Ms = sm;           // m x m: K -> V D^{-1/2}
  double* ev = sm + m * m;   // m
  int* order = reinterpret_cast<int*>(ev + m);
  __shared__ int rotated;
  __shared__ int keff;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    Ms[idx] = 0.5 * (K[idx] + K[j + i * m]);
  }
  __syncthreads();
  psd_eig_scaled(Ms, m, ev, -0.5, rtol, &rotated);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int r = 0;
    for (int i = 0; i < m; ++i) r += (ev[i] > ev[j]) || (ev[i] == ev[j] && i < j);
    order[r] = j;
  }
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int j = 0; j < m; ++j) mx = fmax(mx, ev[j]);
    int r = 0;
    for (int j = 0; j < m; ++j) r += (ev[j] > rtol * mx && ev[j] > 0.0);
    keff = r < k ? r : k;
  }
  __syncthreads();
  const int ke = keff;
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
    const int i = idx % m, r = idx / m;
    SB[i + (long long)r * m] = (r < ke) ? Ms[i + order[r] * m] : 0.0;
  }
  if (threadIdx.x == 0) {
    double lamk = 1.0;
    for (int r = 0; r < k; ++r) {
      D[r] = (r < ke) ? ev[order[r]] : 0.0;
      if (r == ke - 1) lamk = 1.0 + D[r];
    }
    double th = theta_given;
    if (theta_mode == EDA_THETA_LAMBDA_K) th = lamk;
    if (theta_mode == EDA_THETA_MID) th = 0.5 * (lamk + 1.0);
    *theta_out = th;
    for (int r = 0; r < k; ++r) cvec[r] = (r < ke) ? th / (1.0 + D[r]) - 1.0 : 0.0;
    *rank_out = ke;
  }
}

// ---------------------------------------------------------------------------
// Batched PCG vector kernels: one CTA per member (column).
// ---------------------------------------------------------------------------

// Start: bnorm, relres and convergence at x0; r given.  z, p set by caller.
// Item geometry: with item arrays, item j has length n_of[j] at offset
// off_of[j] of the concatenated vectors; without, length n at j*n.
struct ItemGeo {
  const int* n_of;
  const long long* off_of;
};
__device__ __forceinline__ void item_geo(const ItemGeo& ig, int j, int n, int* nj, long long* off) {
  if (ig.n_of) {
    *nj = ig.n_of[j];
    *off = ig.off_of[j];
  } else {
    *nj = n;
    *off = (long long)j * n;
  }
}

template <typename T>
__global__ void pcg_start_kernel(int n, ItemGeo ig, const double* b, const T* r, PcgScalars* sc, int* active,
                                 double tol, int* nactive) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  long long off;
  item_geo(ig, j, n, &n, &off);
  const double* bj = b + off;
  const T* rj = r + off;
  double sb = 0.0, sr = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    sb += bj[g] * bj[g];
    sr += (double)rj[g] * (double)rj[g];
  }
  sb = block_sum<double>(sb, red);
  sr = block_sum<double>(sr, red);
  if (threadIdx.x == 0) {
    const double bn = sqrt(sb);
    sc[j].bnorm = bn;
    sc[j].relres = bn > 0.0 ? sqrt(sr) / bn : 0.0;
    sc[j].iters = 0;
    sc[j].status = EDA_MAXIT;
    sc[j].tolm = 0.0;
    sc[j].errb = __longlong_as_double(0x7ff8000000000000ll);
    const bool done = (bn == 0.0) || (tol > 0.0 && sc[j].relres <= tol);
    if (done) sc[j].status = EDA_CONVERGED;
    active[j] = done ? 0 : 1;
    if (!done) atomicAdd(nactive, 1);
  }
}


template <typename TS, typename TD>
__global__ void convert_kernel(long long count, const TS* s, TD* d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = (TD)s[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <typename TA, typename TB>
cudaError_t gemm_tn(int n, const TA* A, int ka, const TB* B, int mb, double* Cm, int ldc,
                    const int* active_cols, bool sym, cudaStream_t s) {
  if (ka <= 0 || mb <= 0) return cudaSuccess;
  count_launch();
  gemm_tn_kernel<TA, TB><<<dim3(ka, mb), 256, 0, s>>>(n, A, ka, B, mb, Cm, ldc, active_cols, sym ? 1 : 0);
  return cudaGetLastError();
}

template <typename TA, typename TZ>
cudaError_t gemm_nn(int n, const TA* A, int k, int m, const double* Bs, const double* scale, const TZ* R,
                    TZ* Z, const int* active_cols, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int threads = 256;
  count_launch();
  gemm_nn_kernel<TA, TZ><<<dim3((n + threads - 1) / threads, m), threads, (size_t)k * sizeof(double), s>>>(
      n, A, k, Bs, scale, R, Z, active_cols);
  return cudaGetLastError();
}

cudaError_t chol_inv(const double* G, int m, double shift, double* R, double* Rinv, int* status,
                     cudaStream_t s) {
  const size_t smem = (size_t)2 * m * m * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  chol_inv_kernel<<<1, 256, smem, s>>>(G, m, shift, R, Rinv, status);
  return cudaGetLastError();
}

cudaError_t tri_mul(const double* A, const double* B, double* P, int m, cudaStream_t s) {
  const size_t smem = (size_t)3 * m * m * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(tri_mul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  tri_mul_kernel<<<1, 256, smem, s>>>(A, B, P, m);
  return cudaGetLastError();
}

cudaError_t nystrom_core(const double* W, const double* RY, int m, int k, double nu, int theta_mode,
                         double theta_given, double* UT, double* D, double* cvec, double* theta_out,
                         int* status, cudaStream_t s) {
  const size_t smem = (size_t)3 * m * m * sizeof(double) + (size_t)m * sizeof(double) + (size_t)m * sizeof(int);
  cudaError_t e =
      cudaFuncSetAttribute(nystrom_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  nystrom_core_kernel<<<1, 1024, smem, s>>>(W, RY, m, k, nu, theta_mode, theta_given, UT, D, cvec, theta_out,
                                            status);
  return cudaGetLastError();
}

cudaError_t robust_winv(const double* W, int m, double rtol, double* M, cudaStream_t s) {
  const size_t smem = ((size_t)m * m + m) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(robust_winv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  robust_winv_kernel<<<1, 1024, smem, s>>>(W, m, rtol, M);
  return cudaGetLastError();
}

cudaError_t robust_eig(const double* K, int m, int k, double rtol, int theta_mode, double theta_given, double* SB,
                       double* D, double* cvec, double* theta_out, int* rank_out, cudaStream_t s) {
  const size_t smem = ((size_t)m * m + m) * sizeof(double) + (size_t)m * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(robust_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  robust_eig_kernel<<<1, 1024, smem, s>>>(K, m, k, rtol, theta_mode, theta_given, SB, D, cvec, theta_out, rank_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t pcg_start(int n, int m, const double* b, const T* r, PcgScalars* sc, int* active, double tol,
                      int* nactive, cudaStream_t s, const int* n_of, const long long* off_of) {
  count_launch();
  pcg_start_kernel<T><<<m, 256, 0, s>>>(n, ItemGeo{n_of, off_of}, b, r, sc, active, tol, nactive);
  return cudaGetLastError();
}

template <typename TS, typename TD>
cudaError_t convert(long long count, const TS* src, TD* dst, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  convert_kernel<TS, TD><<<(unsigned)blocks, 256, 0, s>>>(count, src, dst);
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t gemm_tn<double, double>(int, const double*, int, const double*, int, double*, int,
                                             const int*, bool, cudaStream_t);
template cudaError_t gemm_tn<float, float>(int, const float*, int, const float*, int, double*, int,
                                           const int*, bool, cudaStream_t);
template cudaError_t gemm_nn<double, double>(int, const double*, int, int, const double*, const double*,
                                             const double*, double*, const int*, cudaStream_t);
template cudaError_t gemm_nn<float, float>(int, const float*, int, int, const double*, const double*,
                                           const float*, float*, const int*, cudaStream_t);
template cudaError_t pcg_start<double>(int, int, const double*, const double*, PcgScalars*, int*, double, int*,
                                       cudaStream_t, const int*, const long long*);
template cudaError_t pcg_start<float>(int, int, const double*, const float*, PcgScalars*, int*, double, int*,
                                      cudaStream_t, const int*, const long long*);
template cudaError_t convert<double, float>(long long, const double*, float*, cudaStream_t);
template cudaError_t convert<float, double>(long long, const float*, double*, cudaStream_t);

}  // namespace eda
