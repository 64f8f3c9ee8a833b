/*
 * eda.h — C ABI of the GB300 (sm_103a) ensemble-of-4D-Var solver library
 * (libeda.so).
 *
 * The library solves, for every member j of an ensemble data assimilation
 * (EDA) with a Lorenz-96 model, the incremental strong-constraint 4D-Var
 * system in the control variable (Section 2.3, Eq. (system with CVT)):
 *
 *     (I + A_j) dz_j = b_j,   A_j = U_B^T G_j^T R^{-1} G_j U_B,
 *                             b_j = U_B^T G_j^T R^{-1} d_j,
 *
 * with a second-level scaled spectral LMP (Section 3.1) built from a Nystrom
 * approximation (Section 3.2.3, Algorithm 1) of the control member's A,
 * sketched with the matrix of right-hand-side differences Gamma
 * (Section 3.2.2, Eq. (Gamma)), and batched preconditioned CG.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an eda_status.  EDA_OK is 0; on any other value
 *   eda_last_error() returns a message.  A member that does not converge is
 *   NOT an error: it is reported in status_out of eda_solve_batch.
 * - Vectors are FP64, member-major: member (or column) c occupies elements
 *   [c*n, (c+1)*n).  Observation-space arrays are FP64, member-major with
 *   p = obs_ptr[n_obs_times] entries per member, ordered by observation step
 *   then by the order of obs_idx.
 * - Array arguments may be HOST or DEVICE memory (the library asks the CUDA
 *   runtime which).  Device arrays are used in place on the handle's stream.
 *   Host arrays are copied through the handle's staging buffers on that
 *   stream; a call that writes a host array synchronises the stream before
 *   returning.  The caller owns every argument array; the handle owns its
 *   internal buffers (trajectory store, right-hand sides, sketch, LMP).
 * - Calls on one handle are not thread-safe; distinct handles are
 *   independent.
 */
#ifndef EDA_H
#define EDA_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define EDA_API __attribute__((visibility("default")))
#else
#define EDA_API
#endif

typedef enum {
  EDA_OK = 0,
  EDA_ERR_INVALID = 1,  /* a size, pointer or option is out of range        */
  EDA_ERR_CUDA = 2,     /* a CUDA runtime call failed                         */
  EDA_ERR_NUMERIC = 3,  /* NaN/Inf in an input, or Cholesky failure after the
                           Appendix B shift retry                             */
  EDA_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up                 */
  EDA_ERR_STATE = 5     /* calls out of order (e.g. solve before set_trajectory) */
} eda_status;

/* precision */
enum { EDA_FP64 = 0, EDA_MIXED = 1 };
/* theta_mode: the scaling of the spectral LMP (Section 3.1) */
enum { EDA_THETA_GIVEN = 0, EDA_THETA_LAMBDA_K = 1, EDA_THETA_MID = 2 };
/* per-member solve status */
enum { EDA_CONVERGED = 0, EDA_MAXIT = 1, EDA_NAN = 2, EDA_BREAKDOWN = 3 };

typedef struct eda_handle eda_handle;

/*
 * Problem definition.  All pointers in this struct are HOST pointers; the
 * library copies what it needs during eda_create.
 *
 *  n, nsteps       state size (n >= 4) and window length N (N >= 1):
 *                  states x_0 .. x_N (Section 2.1).
 *  F, dt           Lorenz-96 forcing and RK4 step (Section 4: F = 8,
 *                  dt = 0.025).
 *  n_obs_times     number of observation steps (>= 1).
 *  obs_steps       [n_obs_times] strictly increasing steps in [0, N].
 *  obs_ptr         [n_obs_times+1] CSR offsets into obs_idx (obs_ptr[0] = 0).
 *  obs_idx         [p] observed variable indices in [0, n), strictly
 *                  increasing within each step: H_t selects them.
 *  rinv            [p] diagonal of R^{-1} (R = sigma_o^2 I in Section 4).
 *  bhalf_w, bhalf_coef
 *                  U_B = U_B^T as the banded symmetric circulant
 *                  (U_B v)_i = sum_{|d|<=w} coef[|d|] v_{(i+d) mod n},
 *                  0 <= w <= (n-1)/2, coef has w+1 entries.
 *  n_members       L + 1 (member 0 is the control, Section 2.2), >= 1.
 *  ell, k          sketch columns (1 <= ell <= min(L, 80, n)) and LMP rank (1 <= k <= ell)
 *                  (Algorithm 1).  ell = 0 disables the LMP.
 *  theta_mode, theta   EDA_THETA_GIVEN uses theta; EDA_THETA_LAMBDA_K uses
 *                  lambda_k(I+A); EDA_THETA_MID uses (lambda_k(I+A)+1)/2
 *                  (Section 3.1).
 *  precision       EDA_FP64: every sweep, vector and scalar in FP64.
 *                  EDA_MIXED: tangent-linear/adjoint sweeps and LMP apply in
 *                  FP32, CG scalars, residual norms and the small Nystrom
 *                  factorisations in FP64, FP64 residual replacement.
 *  ckpt_every      0 stores the whole trajectory; c in [1, 4096] stores the
 *                  states x_0, x_c, x_2c, ... only, and every Hessian-product
 *                  and right-hand-side sweep recomputes each c-step segment
 *                  from its checkpoint on the chip (multi-launch tiles of c
 *                  steps with a halo of 19c + 8; the FP64 stage-state store
 *                  is off).  EDA_ERR_INVALID when no such tiling fits (c too
 *                  large for shared memory).  Checkpointed handles are not
 *                  grouped (eda_group_create).
 *  stream          a cudaStream_t (NULL = the legacy default stream).
 */
typedef struct {
  int n;
  int nsteps;
  double F;
  double dt;
  int n_obs_times;
  const int* obs_steps;
  const int* obs_ptr;
  const int* obs_idx;
  const double* rinv;
  int bhalf_w;
  const double* bhalf_coef;
  int n_members;
  int ell;
  int k;
  int theta_mode;
  double theta;
  int precision;
  int ckpt_every;
  void* stream;
} eda_config;

/* Library version string (static storage). */
EDA_API const char* eda_version(void);

/* Message of the last error on this handle; with h == NULL, of the last
 * failed eda_create or handle-less call on this thread.  Static or
 * handle-owned storage, valid until the next call on the handle. */
EDA_API const char* eda_last_error(const eda_handle* h);

/*
 * Creates a handle for one EDA problem (Section 2.2: L perturbed members and
 * a control) on the current CUDA device.  Validates the configuration
 * (EDA_ERR_INVALID on any out-of-range value or unsorted observation list),
 * copies the observation network and U_B taps to the device and allocates
 * the trajectory store.  *out receives the handle (NULL on failure).
 */
EDA_API int eda_create(const eda_config* cfg, eda_handle** out);

/* Releases every device buffer of the handle.  NULL is accepted. */
EDA_API int eda_destroy(eda_handle* h);

/*
 * Identical-twin generator (Section 4): spins up x_spin0 [n] for `spinup`
 * RK4 steps to the truth x^t_0, integrates the truth over the window and
 * observes it, and forms
 *   x_b,0 = x^t_0 + U_B eta_b[0],      y_0 = H x^t + R^{1/2} eta_o[0],
 *   x_b,j = x_b,0 + U_B eta_b[j],      y_j = y_0 + R^{1/2} eta_o[j]
 * (Section 2.2) for j = 1..L.  eta_b is [(L+1) x n], eta_o [(L+1) x p],
 * standard-normal draws supplied by the caller.  Outputs xb_out
 * [(L+1) x n] and y_out [(L+1) x p]; xt0_out [n] may be NULL.  FP64.
 */
EDA_API int eda_twin(eda_handle* h, const double* x_spin0, int spinup,
                     const double* eta_b, const double* eta_o,
                     double* xb_out, double* y_out, double* xt0_out);

/*
 * Setup of every member (Section 2.1 and 2.2): integrates the nonlinear
 * model from each background xb [(L+1) x n] in FP64, stores the trajectory
 * (or its checkpoints), forms the innovations d_j = y_j - G(x_b,j) from
 * y [(L+1) x p], and the right-hand sides b_j = U_B^T G_j^T R^{-1} d_j by one
 * adjoint sweep per member (FP64).  rhs_out [(L+1) x n] may be NULL.
 * Invalidates any previous sketch and LMP.
 */
EDA_API int eda_set_trajectory(eda_handle* h, const double* xb, const double* y,
                               double* rhs_out);

/*
 * Sketch Y = A Phi of the control member's Hessian (Algorithm 1, first
 * step, with q-1 further power passes when q > 1).  phi [n x ell] is
 * column-major (column c at [c*n, (c+1)*n)); phi == NULL uses
 * Gamma = [b_1 - b_0, ..., b_ell - b_0] (Section 3.2.2, Eq. (Gamma)).
 * y_out [n x ell] (may be NULL) receives A Phi of the last pass.  Requires
 * eda_set_trajectory.  Sweeps in FP64 (EDA_FP64) or FP32 (EDA_MIXED).
 */
EDA_API int eda_sketch(eda_handle* h, const double* phi, int q, double* y_out);

/*
 * Rest of Algorithm 1 in FP64 on the stored sketch: economic QR of Y
 * (CholeskyQR2), W = Phi^T Y, W = C^T C (with the Appendix B shift
 * nu = eps ||Y||_F if the factorisation breaks down), T = R_Y C^{-1}, SVD
 * T = U_T Sigma V_T^T, S = Q_Y U_T, D = Sigma^2, truncated to k; then the
 * LMP coefficients c_i = theta / (1 + D_i) - 1 (Section 3.1).  If the
 * shifted factorisation also breaks down (a numerically rank-deficient
 * sketch), W = Phi^T Y is inverted by a truncated eigendecomposition over
 * its eigenvalues above 1e-12 times the largest, and the range of Y taken
 * from the eigendecomposition of Y^T Y (Appendix B).  That approximation
 * has rank r = the number of eigenvalues kept, so only k_eff = min(k, r)
 * modes are informative: columns k_eff..k-1 of S_k are zero, their D_i = 0
 * and c_i = 0 (the LMP is the identity there), and theta is taken at mode
 * k_eff.  eigvals_out [k] (may be NULL) receives lambda_i(I + A) = 1 + D_i
 * in descending order; s_out [n x k] column-major (may be NULL) receives
 * S_k.  EDA_ERR_NUMERIC if the last CholeskyQR pass of the truncated
 * variant fails.
 */
EDA_API int eda_build_lmp(eda_handle* h, double* eigvals_out, double* s_out);

/*
 * How the last eda_build_lmp went (host outputs, each may be NULL): *path =
 * 0 (Cholesky of W), 1 (Appendix B shift) or 2 (truncated
 * eigendecomposition); *rank = the number of informative LMP modes (k, or
 * k_eff on path 2; k after eda_set_lmp); *shift = nu (0 unless path 1).
 * EDA_ERR_STATE before any LMP.
 */
EDA_API int eda_lmp_info(eda_handle* h, int* path, int* rank, double* shift);

/*
 * Loads a spectral LMP built elsewhere (another process, a previous cycle, a
 * test): s_in [n x k] column-major with orthonormal columns approximating
 * eigenvectors of A, eigvals_in [k] the matching lambda_i(I + A) >= 1 in
 * descending order.  theta follows the handle's theta_mode (Section 3.1).
 * Replaces any LMP from eda_build_lmp.  EDA_ERR_INVALID on a non-finite or
 * out-of-order eigenvalue.
 */
EDA_API int eda_set_lmp(eda_handle* h, const double* s_in, const double* eigvals_in);

/*
 * Batched PCG (Section 2.3) on (I + A_j) dz_j = b_j for every member j, each
 * with its own Hessian, preconditioned by the control member's LMP when
 * use_lmp != 0 (requires eda_build_lmp).  Stops member j when
 * ||r_j|| / ||b_j|| <= tol on the recurrence residual (tol = 0 runs exactly
 * maxit iterations), or after its own maxit-th iteration (the budget is per
 * member, refinement rounds included).  x0 [(L+1) x n] is the
 * initial guess (NULL = 0).  Outputs: dz_out [(L+1) x n], iters_out
 * [L+1] (int), relres_out [L+1] (the FP64 recurrence residual at exit; in
 * EDA_MIXED the FP64 true residual), status_out [L+1] (EDA_CONVERGED,
 * EDA_MAXIT, EDA_NAN, EDA_BREAKDOWN).  Any output may be NULL except dz_out.
 */
EDA_API int eda_solve_batch(eda_handle* h, double tol, int maxit, const double* x0,
                            int use_lmp, double* dz_out, int* iters_out,
                            double* relres_out, int* status_out);

/*
 * Options of eda_solve.  Zero-initialise the struct, then set the fields you
 * need; with every field 0 but maxit it runs exactly maxit iterations.
 *
 *  tol        stop member j when ||r_j|| / ||b_j|| <= tol on the recurrence
 *             residual (the paper's system, Section 2.3); 0 = off.
 *  err_tol    stop member j when ||r_j|| / (||x_j|| - ||r_j||) <= err_tol.
 *             Since every eigenvalue of I + A is >= 1 (Section 2.3),
 *             ||x - x*|| <= ||r|| and ||x*|| >= ||x|| - ||r||, so this is a
 *             certified bound on the relative error ||x_j - x*_j|| /
 *             ||x*_j||; the FP64 true residual b - (I + A) x confirms it at
 *             exit (members whose true bound misses it go on).  0 = off.
 *             With both tol and err_tol set, a member stops when both hold.
 *  maxit      iteration budget per member (refinement rounds included).
 *  use_lmp    precondition with the LMP (requires eda_build_lmp or
 *             eda_set_lmp).
 *  split      1: the split preconditioner P_theta = U_theta U_theta^T
 *             (Section 3.1, Eq. (lmp)): CG on U H U y = U b, x = U y, which
 *             has the same iterates as PCG with P_theta in exact arithmetic;
 *             its stopping test is on its own residual U (b - H x) relative
 *             to U b.  Requires use_lmp, EDA_FP64 and lmp_kind 0 (an error
 *             in U v is multiplied by the leading eigenvalues of H before U
 *             damps them again); err_tol must be 0.
 *  lmp_kind   0: the LMP on CUDA cores, in FP64 (EDA_FP64) or FP32
 *             (EDA_MIXED); 1: on tensor cores, S and the vectors split into
 *             BF16 high and low parts, three products with FP32
 *             accumulation (relative error of the LMP correction ~1e-5);
 *             k <= 128.
 *  x0         [(L+1) x n] initial guess (host or device), NULL = 0.
 *  cost_out   [(L+1) x (maxit+1)] FP64 (host or device) or NULL: the
 *             quadratic cost J(x_i) = 1/2 x_i^T (I + A) x_i - b^T x_i of every
 *             iterate (Section 2, Eq. (2) up to its constant), i = 0 first,
 *             from the recurrence residual (J = -x^T (b + r) / 2); NaN after
 *             a member's last iteration.
 */
typedef struct {
  double tol;
  double err_tol;
  int maxit;
  int use_lmp;
  int split;
  int lmp_kind;
  const double* x0;
  double* cost_out;
} eda_solve_opts;

/*
 * Batched PCG with options (see eda_solve_opts); otherwise as
 * eda_solve_batch.  err_bound_out [L+1] (may be NULL) receives the certified
 * bound ||r|| / (||x|| - ||r||) of the FP64 true residual at exit (NaN when
 * no true residual was taken: EDA_FP64 with err_tol = 0 and err_bound_out
 * NULL takes none); relres_out then holds the true relative residual.
 * EDA_ERR_INVALID on a NULL opts or dz_out, a negative tolerance or maxit.
 */
EDA_API int eda_solve(eda_handle* h, const eda_solve_opts* opts, double* dz_out, int* iters_out,
                      double* relres_out, double* err_bound_out, int* status_out);

/*
 * The LMP on caller vectors (Section 3.1): Z[c] = R[c] + S_k diag(coef)
 * S_k^T R[c] for c < ncol with coef the coefficients of which = 0: P_theta
 * (theta / (1 + lambda_i) - 1), 1: U_theta (sqrt(theta) (1 + lambda_i)^{-1/2}
 * - 1), 2: U_theta^{-1} (1 / (1 + those) - 1).  kind as lmp_kind of
 * eda_solve_opts.  R, Z [ncol x n] FP64, host or device (Z may equal R).
 * Requires eda_build_lmp or eda_set_lmp.  EDA_ERR_TIMEOUT if a bounded wait
 * on the tensor core gave up (outputs then incomplete).
 */
EDA_API int eda_lmp_apply(eda_handle* h, int which, int kind, int ncol, const double* R, double* Z);

/*
 * A spectral LMP from Ritz pairs of one member's Hessian (Section 3: the
 * limited-memory preconditioners built from the Ritz pairs of an earlier CG
 * run, the design the paper's randomized LMP is set against).  Runs `iters`
 * iterations of CG without preconditioner from x0 = 0 on (I + A_m) x = b,
 * A_m the Hessian term of member m = `member` (FP64 sweeps, one Hessian
 * product per iteration, a host round trip per iteration); b [n] FP64, host
 * or device (caller-owned, read only), or NULL for member m's own right-hand
 * side from eda_set_trajectory.  Takes the Lanczos basis v_j = (-1)^j r_j /
 * |r_j| and the tridiagonal T = V^T (I + A_m) V from CG's coefficients
 * (T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T[j][j+1] = sqrt(beta_j) /
 * alpha_j), its eigenpairs (theta_i, y_i), and installs the k leading Ritz
 * pairs (theta_i, V y_i) as the handle's LMP, as eda_set_lmp would (theta
 * mode of the handle; Ritz values below 1 by rounding taken as 1).  The
 * basis is not reorthogonalised.  ritz_out (host, may be NULL) receives all
 * `iters` Ritz values in descending order.  Requires eda_set_trajectory;
 * EDA_ERR_INVALID unless 0 <= member < L+1 and k <= iters <= min(256, n);
 * EDA_ERR_NUMERIC on a zero or non-finite b, a CG breakdown, or if CG
 * converges first.  Synchronises the stream.
 */
EDA_API int eda_ritz_lmp(eda_handle* h, int member, int iters, const double* b, double* ritz_out);

/*
 * Control-variable transform (Section 2.3, Eq. (system with CVT)): OUT[c] =
 * U_B V[c] for c < ncol, U_B the handle's symmetric banded circulant square
 * root of B (taps bhalf_coef).  Maps solutions dz_j of eda_solve_batch to
 * analysis increments dx_j = U_B dz_j, and builds B-shaped sketch matrices
 * (U_B Psi, B Psi = U_B U_B Psi).  V, OUT [ncol x n] FP64, host or device
 * (caller-owned, not overlapping); a host OUT is complete on return.
 * EDA_ERR_INVALID on ncol < 0 or a NULL buffer with ncol > 0.
 */
EDA_API int eda_bhalf_apply(eda_handle* h, int ncol, const double* V, double* OUT);

/*
 * Batched Hessian-vector products (Section 2.3, Eq. (system with CVT)):
 * HV[c] = (include_identity ? V[c] : 0) + A_{m(c)} V[c] for c < ncol, with
 * m(c) = member_of_col[c] in [0, L] choosing the trajectory (the
 * linearisation state).  V, HV are [ncol x n].  Requires
 * eda_set_trajectory.  Sweeps in FP64 (EDA_FP64) or FP32 (EDA_MIXED).
 * A member index outside [0, L]: EDA_ERR_INVALID when member_of_col is
 * host memory (checked before any work); when it is device memory the
 * kernel checks it, reads no trajectory for that column and writes NaN to
 * its row of HV.
 */
EDA_API int eda_hvp(eda_handle* h, const int* member_of_col, int ncol, const double* V,
                    double* HV, int include_identity);

/*
 * Autotuner of the sweep tiling: for the stored trajectories, times the
 * batched member Hessian-vector sweep (all L+1 members) for every tiling
 * that fits -- thread-block cluster size 1..8 (CTAs per vector) and halo
 * refresh period K in {2, 4, 8, 16} steps (FP64 sweeps also K = 1), run
 * lengths, warp-tiled and multi-launch tilings -- and keeps the fastest for all
 * later sweeps of the handle.  which: bit 0 tunes the FP64 sweep, bit 1 the
 * FP32 sweep (EDA_MIXED only); 0 = the sweeps of the handle's precision.
 * *best_ms_out (may be NULL) = sum of the chosen tilings' mean times (ms).
 * Requires eda_set_trajectory.  Synchronises the stream.
 */
EDA_API int eda_autotune(eda_handle* h, int which, double* best_ms_out);

/*
 * The tiling the Hessian-product sweeps of one precision (fp64 != 0: FP64,
 * else FP32) use at this point (after eda_autotune, the autotuned one).
 * info[8] (host, caller-owned) receives: [0] kind (0 thread-block cluster,
 * 1 multi-launch tiles of K steps, 2 warp-tiled), [1] CTAs per state vector
 * (cluster size or tiles), [2] threads per CTA, [3] values per thread (C),
 * [4] halo refresh period K (steps), [5] halo width HL (points, each end),
 * [6] owned points per CTA, [7] dynamic shared memory per CTA (bytes).
 * EDA_ERR_INVALID if fp64 == 0 on an FP64 handle; no device work.
 */
EDA_API int eda_sweep_plan(eda_handle* h, int fp64, int* info);

/*
 * Tilings of the persistent PCG's convergence tail (the solve of Section 2.3
 * run as one launch per phase; not in the paper).  While many members are
 * active the solve runs on the tiling above; a tail tiling of level R serves
 * once at most R members remain active and spreads each over more CTAs: the
 * running launch ends at the iteration boundary after the active count falls
 * to R (every member's PCG state stays on the device) and the solve goes on
 * in a launch on the tail tiling, with the same iterates up to the rounding
 * order of the reductions.  eda_autotune chooses them (active counts falling
 * by an eighth at a time from 7(L+1)/8 to 1; a level is kept where its
 * tiling's Hessian-product sweep beats the main tiling's by more than 7 %)
 * and replaces any set before.
 *
 * eda_tail_plans: *count receives the number of tail tilings of one
 * precision (fp64 != 0: FP64 sweeps, else FP32); levels[i] (may be NULL) and
 * info[8i .. 8i+7] (may be NULL; as in eda_sweep_plan) describe the first
 * min(cap, count), in decreasing level.  Host arrays, caller-owned.
 *
 * eda_set_tail_plan: level in [1, L+1] installs (or replaces, at an equal
 * level) the thread-block cluster tiling of cs CTAs per member, halo refresh
 * period K and C values per thread (0: the main tiling's); level 0 removes
 * every tail tiling of that precision.  EDA_ERR_INVALID when the main tiling
 * is not a cluster tiling (multi-launch, warp-tiled or checkpointed), no
 * tiling of that shape fits, or the persistent PCG cannot run on it.
 * Synchronises the stream.
 */
EDA_API int eda_tail_plans(eda_handle* h, int fp64, int cap, int* count, int* levels, int* info);
EDA_API int eda_set_tail_plan(eda_handle* h, int fp64, int level, int cs, int K, int C);

/*
 * Host-only planning query (no handle, no device work): the tiling the
 * library would use for a Hessian-product sweep of state size n, FP64
 * (fp64 != 0) or FP32, banded circulant half-width w and halo refresh period
 * K.  kind 0: thread-block clusters of exactly cs CTAs with C values per
 * thread (C = 0: the default run length); kind 1: multi-launch tiles of K
 * steps with `threads` threads per CTA (0: the default; C must be 0); kind 2:
 * warp-tiled, clusters of cs CTAs, C values per lane; kind 3: multi-launch
 * tiles for a trajectory checkpointed every K steps (ckpt_every = K; info[0]
 * then reports kind 1).  info[8] (host,
 * caller-owned) as in eda_sweep_plan.  EDA_ERR_INVALID when no tiling of
 * that shape fits (or an argument is out of range).
 */
EDA_API int eda_plan_tiling(int n, int fp64, int w, int kind, int cs, int threads, int K, int C, int* info);

/*
 * Tracing: process-wide number of CUDA kernels the library has launched
 * (every handle, every entry point) since it was loaded.  No device work.
 */
EDA_API long long eda_kernel_launches(void);

/*
 * Tracing of the Hessian-product sweeps of one handle (eda_hvp, the sketch,
 * the PCG of eda_solve_batch, the FP64 true residuals): with enable = e > 0,
 * one later sweep in e (the first, then every e-th) is bracketed by a pair
 * of CUDA events on the handle's stream and the columns it computed (the
 * active members, counted on the device) are summed.  eda_trace(h, e) starts
 * a new record (zeroing the totals); eda_trace(h, 0) stops recording and
 * keeps them.  A traced sweep adds one one-thread kernel and two event
 * records to the stream.  EDA_ERR_INVALID if enable < 0.
 */
EDA_API int eda_trace(eda_handle* h, int enable);
/*
 * Totals of the record (host outputs, each may be NULL): for the FP64
 * sweeps (fp64 != 0) or the FP32 sweeps, *sweeps = sweeps recorded,
 * *columns = columns they computed, *ms = summed event time.  Synchronises
 * the stream.
 */
EDA_API int eda_trace_read(eda_handle* h, int fp64, long long* sweeps, long long* columns, double* ms);

/*
 * Tracing: times `reps` launches of the batched Hessian-vector sweep that the
 * PCG of eda_solve_batch issues (all L+1 members, each on its own
 * trajectory, inputs from the handle's current direction vectors) with CUDA
 * events on the handle's stream, after one untimed launch.  fp64 != 0 times
 * the FP64 sweep, otherwise the sweep of the handle's precision.
 * *ms_out = mean milliseconds per launch.  Requires eda_set_trajectory.
 * Synchronises the stream.
 */
EDA_API int eda_time_hvp_sweep(eda_handle* h, int reps, int fp64, double* ms_out);

/*
 * eda_hvp for callers that must not allocate device memory while they run
 * (the paper has no counterpart: it is an interface for callers).  Such
 * callers include a host thread capturing a CUDA graph in global mode, where
 * cudaMalloc is illegal; an assimilation cycle confined to a preallocated
 * memory budget; a latency-critical loop that cannot afford the device
 * synchronisation an allocation may cause.  eda_hvp may allocate (it grows
 * the handle's observation stash and stages host arrays); this variant
 * computes the same products with no allocation at all:
 *  - member_of_col, V and HV must be device memory (EDA_ERR_INVALID otherwise);
 *    a member index outside [0, L] gives a NaN row of HV (as in eda_hvp);
 *  - its scratch, the per-column observation stash, is a fixed 32 MiB
 *    __device__ array compiled into the library (held by every device that
 *    loads it until the process exits): ncol * p must not exceed
 *    eda_hvp_noalloc_capacity(precision == EDA_FP64) entries, or the call
 *    fails with EDA_ERR_INVALID before any work (split the columns);
 *  - the first call on a device looks up the array's device address (no
 *    allocation); make that first call before any stream capture.  Host
 *    threads may make their first calls concurrently (the cached address
 *    is published atomically);
 *  - every call on a device shares the array: calls that overlap on the GPU
 *    (other streams, other handles) race; calls on one stream do not.  The
 *    stash needs no clearing (each entry is written before it is read).
 */
EDA_API int eda_hvp_noalloc(eda_handle* h, const int* member_of_col, int ncol, const double* V,
                            double* HV, int include_identity);
/* Stash entries the eda_hvp_noalloc scratch holds (FP64 if fp64 != 0, else FP32). */
EDA_API long long eda_hvp_noalloc_capacity(int fp64);

/* ------------------------------------------------------------------------
 * Uneven batching (not in the paper, which solves one EDA at a time): a group
 * of independent EDA problems -- each its own handle, with its own n, window,
 * member count, observation network and U_B, all of one precision and on one
 * stream -- whose sweeps run as single launches over all problems (one per
 * thread-block shape), whose PCG vector updates and LMP applies run as
 * batched launches over every (problem, member), and whose PCG iteration is
 * captured once in a CUDA graph and replayed until every member converges.
 * The handles stay owned by the caller and must outlive the group.
 * ---------------------------------------------------------------------- */
typedef struct eda_group eda_group;

/* Groups count >= 1 handles.  EDA_ERR_INVALID if they differ in precision
 * or stream, or a problem does not fit the sweep tiling. */
EDA_API int eda_group_create(eda_handle* const* handles, int count, eda_group** out);
EDA_API int eda_group_destroy(eda_group* g);
/* Message of the group's last error (static or group-owned storage). */
EDA_API const char* eda_group_last_error(const eda_group* g);
/* eda_set_trajectory of every problem: xb[i] [(L_i+1) x n_i], y[i]
 * [(L_i+1) x p_i] (host array of per-problem pointers, each host or device). */
EDA_API int eda_group_set_trajectories(eda_group* g, const double* const* xb, const double* const* y);
/* Gamma sketch Y = A Gamma of every problem's control Hessian (Algorithm 1,
 * q = 1): all sketch columns of all problems in one launch per bucket. */
EDA_API int eda_group_sketch(eda_group* g);
/* The rest of Algorithm 1 and the LMP of every problem (eda_build_lmp). */
EDA_API int eda_group_build_lmp(eda_group* g);
/* Autotuner of the group's tile shapes: for every problem, tiles of 1 or 2
 * times the fewest CTAs per member that fit, and halo refresh periods K in
 * {2, 4, 8, 16}.  Times the batched member sweep of every resulting bucket
 * (problems of one cluster size and power-of-two CTA size, launched
 * together) alone on the device, charges each problem its share of its
 * bucket's time (by members x n x window), and keeps each problem's cheapest
 * shape and period.  *best_ms_out (may be NULL) = mean time of the tuned
 * batched sweep (ms). */
EDA_API int eda_group_autotune(eda_group* g, double* best_ms_out);
/* Batched PCG of every member of every problem (as eda_solve_batch, x0 = 0;
 * maxit is a budget per member, so one hard problem does not cut the others
 * short).
 * dz_out[i] [(L_i+1) x n_i] per problem (host array of pointers, each host or
 * device, NULL entries skipped; dz_out itself may be NULL); iters_out,
 * relres_out, status_out [sum_i (L_i+1)] concatenated in problem order (host
 * or device, may be NULL).  Synchronises the stream. */
EDA_API int eda_group_solve(eda_group* g, double tol, int maxit, int use_lmp, double* const* dz_out,
                            int* iters_out, double* relres_out, int* status_out);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper): a periodic 1-D convolutional
 * network mapping (member right-hand side b_j, control solution dz_0) to a
 * guess of the member solution dz_j, used only as the initial iterate x0 of
 * eda_solve_batch, which still runs to the same tolerance (so the plain
 * solve still decides the error).
 *
 * Network: channels 2 -> H -> H -> H -> 1, kernel 5 with periodic wrap (tap t
 * reads position i + t - 2 mod n), GELU (erf form) after layers 1-3; inputs
 * [b_j / s_b, dz_0 / s_z] with s_b, s_z the training-set RMS of b and dz_0;
 * guess = dz_0 + s_z * out.  Parameters: FP32 masters, flat, per layer the
 * weights [out][in][5] then the biases; every product uses the weights
 * rounded to BF16, activations and accumulation are FP32 (with 64 hidden
 * channels the 64 -> 64 convolutions run on the tensor cores, each FP32
 * activation split exactly into three BF16 parts; EDA_WS_TC=0 keeps them on
 * CUDA cores; EDA_ERR_TIMEOUT if a bounded wait for the tensor cores gives
 * up).  Training: mean
 * squared error of (guess - dz_j) / s_z, AdamW (beta 0.9/0.999, eps 1e-8,
 * decoupled weight decay).  Samples are [count x n] FP64 arrays (host or
 * device).  Calls on one network are not thread-safe.
 * ---------------------------------------------------------------------- */
typedef struct eda_ws eda_ws;

/* n >= 5 periodic points, 1 <= hidden <= 64 channels, max_batch samples per
 * forward/backward pass; parameters start at zero (set them before use). */
EDA_API int eda_ws_create(int n, int hidden, int max_batch, void* stream, eda_ws** out);
EDA_API int eda_ws_destroy(eda_ws* w);
EDA_API const char* eda_ws_last_error(const eda_ws* w);
/* Number of FP32 parameters (0 for NULL). */
EDA_API long long eda_ws_num_params(const eda_ws* w);
/* He initialisation from standard-normal draws [num_params] FP64 (host or
 * device; one per parameter in the flat layout): weights of a layer with ci
 * input channels = draw * sqrt(2 / (5 ci)), biases 0; resets the AdamW
 * moments. */
EDA_API int eda_ws_init(eda_ws* w, const double* draws);
/* Loads / stores the flat FP32 parameters (host or device); loading resets
 * the AdamW moments.  Together with the scales this is the saved model. */
EDA_API int eda_ws_set_params(eda_ws* w, const float* params);
EDA_API int eda_ws_get_params(eda_ws* w, float* params);
/* Input scales s_b, s_z (> 0); eda_ws_train sets them from its data when
 * they are unset. */
EDA_API int eda_ws_set_scales(eda_ws* w, double s_b, double s_z);
EDA_API int eda_ws_get_scales(const eda_ws* w, double* s_b, double* s_z);
/* Mean loss over count <= max_batch samples and its gradient w.r.t. the
 * parameters (grad_out [num_params] FP32, host or device, may be NULL);
 * no update.  Requires the scales. */
EDA_API int eda_ws_loss_grad(eda_ws* w, const double* rhs, const double* ctrl, const double* sol, int count,
                             double* loss_out, float* grad_out);
/* epochs passes of AdamW over count samples in batches of <= max_batch; order
 * [epochs x count] sample permutation (host or device; NULL = sequential).
 * loss_out [epochs] (host, may be NULL) = mean batch loss per epoch. */
EDA_API int eda_ws_train(eda_ws* w, const double* rhs, const double* ctrl, const double* sol, int count,
                         int epochs, int batch, double lr, double weight_decay, const int* order,
                         double* loss_out);
/* out [count x n] = the network's guesses of dz_j (host or device). */
EDA_API int eda_ws_infer(eda_ws* w, const double* rhs, const double* ctrl, int count, double* out);

/*
 * Host helper: taps of U_B for a Gaussian correlation
 * B = sigma_b^2 exp(-d^2 / (2 L^2)) on the circle of n points:
 * coef[d] = sigma_b (2 / (pi L^2))^{1/4} exp(-d^2 / L^2) for
 * d <= w = min((n-1)/2, floor(L sqrt(ln 1e17))).  Writes w+1 taps to
 * taps_out (capacity max_taps) and w to *w_out.  No device work.
 */
EDA_API int eda_bhalf_gaussian(int n, double length_scale, double sigma_b,
                               double* taps_out, int max_taps, int* w_out);

#ifdef __cplusplus
}
#endif
#endif /* EDA_H */
