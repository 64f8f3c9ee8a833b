"""Plain, slow, FP64 CPU oracle for the ensemble-of-4D-Var hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path (``paper_2605_23571_gb300``) and imports nothing from it.

Every function follows a passage of the paper (Dauzickaite, Gurol,
Destouches, Berre, Weaver, "Accelerating an ensemble of variational data
assimilations with randomized preconditioning"):

* Lorenz-96 tendency and RK4 step ........ Section 4 (model ODE, periodic
  boundary, F = 8, fourth-order Runge-Kutta, dt = 0.025)
* tangent linear / adjoint of that step ... Section 2.1 (G is the Jacobian of
  the generalized observation operator linearised around the background
  trajectory) — realised as the exact derivative of the discrete RK4 step and
  its exact transpose
* B^{1/2} and the control-variable transform  Section 2.3, Eq. (first-level
  preconditioning) and Eq. (system with CVT): (I + A) dz = U_B^T G^T R^{-1} d
* ensemble perturbations .................. Section 2.2 (y_j = y + U_R eta_o,
  x_b,j = x_b + U_B eta_b) and Section 4 (identical twin)
* RHS differences Gamma ................... Section 3.2.2, Eq. (Gamma)
* q-pass Nystrom approximation ............ Section 3.2.3, Algorithm 1
  (shift fallback: Appendix B)
* scaled spectral LMP ..................... Section 3.1 (P_theta, choices of
  theta)
* preconditioned CG ....................... Section 2.3 (CG on the SPD system)
* Ritz pairs from CG (Lanczos) ............ Section 3 (spectral LMPs from the
  Ritz pairs of an earlier CG run)

Parity status: every function here is pinned by a test in
``tests/test_oracle_*.py`` against something other than itself (closed forms,
invariants, finite differences, brute force, library routines on tiny
inputs).  The PCG iteration counts the paper only plots are "parity
unpinned": the paper prints no numbers for them.  Function -> pin:

* l96_tendency ....... fixed point x = F (model), the paper's index form,
                       energy identity of the advection term
* rk4_step, trajectory  local error order 5 against scipy's DOP853
* jac_apply, tl_step . Taylor test (remainder ratio -> 4)
* jacT_apply, adj_step  entrywise transpose; dot-product tests per step and
                       over the window (1e-12)
* bhalf_taps/apply ... closed-form Gaussian taps (golden file); U_B U_B
                       against the Gaussian correlation
* twin, obs_gather ... enter every pin below through the observations;
                       Gamma covariance A + A^2 on a linear twin
* innovations, rhs ... minus the central-difference gradient of the
                       nonlinear cost at dz = 0 (test_rhs_is_minus_...)
* apply_A, hvp, dense_A  finite-difference Hessian of the nonlinear model,
                       circulant closed form at the fixed point, symmetry,
                       eigenvalues >= 1 and the unit cluster
* cost_J ............. J(x) - J(x*) = 1/2 |x - x*|_H^2; history of pcg
                       never increases and ends at J(x_K)
* nystrom ............ full-rank recovery, exact low rank, Phi -> Phi G
                       invariance, power pass, shift and truncated-EVD
                       variants against dense A Phi (Phi^T A Phi)^+ Phi^T A
* theta_value, lmp_coeffs, lmp_apply  exact eigenpairs map the k targeted
                       eigenvalues to theta, the rest unchanged
* pcg ................ dense direct solve (1e-10), with the LMP, from an
                       initial guess x0 (and CG from x0 = x0 + CG on the
                       shifted residual), a-priori bound |e| <= |r|
* lmp_split_coeffs, pcg_split  U U = P_theta and U = U^T on dense matrices;
                       the split iterates equal pcg's (nested Krylov spaces
                       U K(U H U, U b) = K(P H, P b)) and converge to the
                       dense solution
* lanczos_cg ......... V^T V = I and V^T H V = T on an explicit H; with
                       iters = n the Ritz values are eigh(H)'s; the Lanczos
                       residual identity |H s - theta s| = eta |y_last|

Conventions (readings of the paper where it is silent):
* states x_0..x_N on the window; observation steps are given explicitly and
  may include any t in [0, N];
* B^{1/2} is a banded symmetric circulant defined by its taps c_0..c_w (the
  Gaussian square root of a Gaussian correlation of length L, truncated where
  the taps fall below 1e-17 c_0), so U_B = U_B^T and B := U_B U_B exactly;
* R = sigma_o^2 I, R^{-1} passed as a per-observation diagonal.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Lorenz-96 (Section 4, model ODE with periodic boundary)
# ---------------------------------------------------------------------------


def l96_tendency(x, F):
    """dX_j/dt = -X_{j-2} X_{j-1} + X_{j-1} X_{j+1} - X_j + F, indices mod n.

    ``np.roll(x, s)[j] = x[j - s]`` on the last axis.
    """
    xm2 = np.roll(x, 2, axis=-1)
    xm1 = np.roll(x, 1, axis=-1)
    xp1 = np.roll(x, -1, axis=-1)
    return -xm2 * xm1 + xm1 * xp1 - x + F


def rk4_stages(x, F, dt):
    """Stage states X1..X4 of the classical RK4 step and the four slopes."""
    k1 = l96_tendency(x, F)
    X2 = x + 0.5 * dt * k1
    k2 = l96_tendency(X2, F)
    X3 = x + 0.5 * dt * k2
    k3 = l96_tendency(X3, F)
    X4 = x + dt * k3
    k4 = l96_tendency(X4, F)
    return (x, X2, X3, X4), (k1, k2, k3, k4)


def rk4_step(x, F, dt):
    """One classical fourth-order Runge-Kutta step of the model."""
    _, (k1, k2, k3, k4) = rk4_stages(x, F, dt)
    return x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def trajectory(x0, F, dt, nsteps):
    """States x_0..x_N; shape (..., N+1, n)."""
    xs = [np.asarray(x0, dtype=np.float64)]
    for _ in range(nsteps):
        xs.append(rk4_step(xs[-1], F, dt))
    return np.stack(xs, axis=-2)


def jac_apply(X, v):
    """J(X) v for the tendency: the derivative of l96_tendency at X along v."""
    Xm2, Xm1, Xp1 = np.roll(X, 2, -1), np.roll(X, 1, -1), np.roll(X, -1, -1)
    vm2, vm1, vp1 = np.roll(v, 2, -1), np.roll(v, 1, -1), np.roll(v, -1, -1)
    return (vp1 - vm2) * Xm1 + (Xp1 - Xm2) * vm1 - v


def jacT_apply(X, w):
    """J(X)^T w: the transpose of jac_apply, entry by entry.

    Row i of J has x_{i-1} at column i+1, -x_{i-1} at column i-2,
    (x_{i+1} - x_{i-2}) at column i-1 and -1 at column i; collecting the
    entries of column j gives the four terms below.
    """
    Xm2, Xm1 = np.roll(X, 2, -1), np.roll(X, 1, -1)
    Xp1, Xp2 = np.roll(X, -1, -1), np.roll(X, -2, -1)
    wm1, wp1, wp2 = np.roll(w, 1, -1), np.roll(w, -1, -1), np.roll(w, -2, -1)
    return Xm2 * wm1 + (Xp2 - Xm1) * wp1 - Xp1 * wp2 - w


def tl_step(x, dx, F, dt):
    """Exact derivative of rk4_step at x along dx (tangent-linear model)."""
    (X1, X2, X3, X4), _ = rk4_stages(x, F, dt)
    dk1 = jac_apply(X1, dx)
    dk2 = jac_apply(X2, dx + 0.5 * dt * dk1)
    dk3 = jac_apply(X3, dx + 0.5 * dt * dk2)
    dk4 = jac_apply(X4, dx + dt * dk3)
    return dx + (dt / 6.0) * (dk1 + 2.0 * dk2 + 2.0 * dk3 + dk4)


def adj_step(x, lam, F, dt):
    """Exact transpose of tl_step at x applied to lam (adjoint model).

    Reverse-mode of the four stage recurrences of tl_step.
    """
    (X1, X2, X3, X4), _ = rk4_stages(x, F, dt)
    a4 = (dt / 6.0) * lam
    a3 = (dt / 3.0) * lam
    a2 = (dt / 3.0) * lam
    a1 = (dt / 6.0) * lam
    out = lam.copy()
    g4 = jacT_apply(X4, a4)
    out = out + g4
    a3 = a3 + dt * g4
    g3 = jacT_apply(X3, a3)
    out = out + g3
    a2 = a2 + 0.5 * dt * g3
    g2 = jacT_apply(X2, a2)
    out = out + g2
    a1 = a1 + 0.5 * dt * g2
    g1 = jacT_apply(X1, a1)
    return out + g1


# ---------------------------------------------------------------------------
# Background-error covariance square root (Section 2.3 / Section 4)
# ---------------------------------------------------------------------------


def bhalf_taps(n, length_scale, sigma_b, tol=1e-17):
    """Taps c_0..c_w of U_B, the square root (under periodic convolution) of
    a Gaussian correlation B = sigma_b^2 exp(-d^2 / (2 L^2)).

    The square root of a Gaussian kernel of length L under convolution is the
    Gaussian of length L / sqrt(2) scaled to unit-normalised product:
    c_d = sigma_b (2 / (pi L^2))^{1/4} exp(-d^2 / L^2).  On the integer grid,
    by Poisson summation, (U_B U_B)_{0,d} = sigma_b^2 exp(-d^2/(2L^2))
    (1 + O(exp(-pi^2 L^2 / 2))).  The taps are truncated at the largest d with
    c_d >= tol c_0 and at (n-1)/2, so that the banded form is exactly a
    symmetric circulant.  (A square root taken through the DFT of the sampled
    correlation is not used: the square root of its ~1e-16 high-frequency
    eigenvalues turns FFT rounding into ~1e-8 noise in the taps.)
    """
    L = float(length_scale)
    wcut = int(np.floor(L * np.sqrt(-np.log(tol))))
    w = max(0, min((n - 1) // 2, wcut))
    d = np.arange(w + 1, dtype=np.float64)
    return sigma_b * (2.0 / (np.pi * L * L)) ** 0.25 * np.exp(-(d * d) / (L * L))


def bhalf_apply(v, taps):
    """(U_B v)_i = sum_{|d| <= w} c_|d| v_{(i+d) mod n} on the last axis."""
    out = taps[0] * v
    for d in range(1, len(taps)):
        out = out + taps[d] * (np.roll(v, d, -1) + np.roll(v, -d, -1))
    return out


def bhalf_dense(n, taps):
    """U_B as an explicit n x n matrix (small n only)."""
    return bhalf_apply(np.eye(n), taps)


# ---------------------------------------------------------------------------
# Twin experiment and ensemble perturbations (Sections 2.2 and 4)
# ---------------------------------------------------------------------------


def obs_gather(spec, states):
    """H_t x_t for every observation step, concatenated: shape (..., p).

    ``states`` has shape (..., N+1, n).
    """
    out = []
    for j, t in enumerate(spec.obs_steps):
        idx = spec.obs_idx[spec.obs_ptr[j]: spec.obs_ptr[j + 1]]
        out.append(states[..., int(t), :][..., idx])
    return np.concatenate(out, axis=-1)


def twin(spec, dr, taps):
    """Identical twin: spun-up truth, control background, perturbed members.

    Returns (x_truth0, xb (L+1, n), y (L+1, p)).  Member 0 is the control.
    """
    F, dt = spec.F, spec.dt
    x = F + spec.spin_sigma * dr.eta_spin
    for _ in range(spec.spinup):
        x = rk4_step(x, F, dt)
    return twin_from_truth(spec, dr, taps, x)


def twin_from_truth(spec, dr, taps, xt0):
    """The twin of ``twin`` from a given spun-up truth x^t_0: truth over the
    window, observations, control background and perturbed members.

    Returns (x_truth0, xb (L+1, n), y (L+1, p)).
    """
    F, dt = spec.F, spec.dt
    xt0 = np.asarray(xt0, dtype=np.float64)
    truth = trajectory(xt0, F, dt, spec.nsteps)
    sig_o = 1.0 / np.sqrt(spec.rinv)
    y0 = obs_gather(spec, truth) + sig_o * dr.eta_o[0]
    xb0 = xt0 + bhalf_apply(dr.eta_b[0], taps)
    L1 = spec.n_members
    xb = np.empty((L1, spec.n))
    y = np.empty((L1, spec.p))
    xb[0] = xb0
    y[0] = y0
    for j in range(1, L1):
        xb[j] = xb0 + bhalf_apply(dr.eta_b[j], taps)
        y[j] = y0 + sig_o * dr.eta_o[j]
    return xt0, xb, y


# ---------------------------------------------------------------------------
# Innovations, RHS, Hessian-vector products (Section 2.1, Eq. (system with CVT))
# ---------------------------------------------------------------------------


def member_trajectories(spec, xb):
    """Nonlinear trajectories of every member, shape (M, N+1, n)."""
    return trajectory(xb, spec.F, spec.dt, spec.nsteps)


def innovations(spec, traj, y):
    """d_j = y_j - G(x_b,j), the obs-space departures of each member."""
    return y - obs_gather(spec, traj)


def _obs_slices(spec):
    return {int(t): spec.obs_idx[spec.obs_ptr[j]: spec.obs_ptr[j + 1]]
            for j, t in enumerate(spec.obs_steps)}, \
           {int(t): slice(int(spec.obs_ptr[j]), int(spec.obs_ptr[j + 1]))
            for j, t in enumerate(spec.obs_steps)}


def adjoint_sweep(spec, traj, forcing):
    """sum_t M_{0->t}^T H_t^T forcing_t, by one backward sweep.

    ``traj``: (M, N+1, n); ``forcing``: (M, p) obs-space vectors.
    """
    idx_of, sl_of = _obs_slices(spec)
    M = traj.shape[0]
    lam = np.zeros((M, spec.n))
    for t in range(spec.nsteps, -1, -1):
        if t < spec.nsteps:
            lam = adj_step(traj[:, t, :], lam, spec.F, spec.dt)
        if t in idx_of:
            np.add.at(lam, (slice(None), idx_of[t]), forcing[:, sl_of[t]])
    return lam


def tangent_sweep(spec, traj, dx0):
    """[H_t M_{0->t} dx0]_t concatenated over obs steps: shape (M, p)."""
    idx_of, _ = _obs_slices(spec)
    out = []
    dx = dx0.copy()
    for t in range(0, spec.nsteps + 1):
        if t > 0:
            dx = tl_step(traj[:, t - 1, :], dx, spec.F, spec.dt)
        if t in idx_of:
            out.append(dx[:, idx_of[t]])
    return np.concatenate(out, axis=-1) if out else np.zeros((dx0.shape[0], 0))


def rhs(spec, traj, d, taps):
    """b_j = U_B^T G_j^T R^{-1} d_j (Eq. (system with CVT), right-hand side)."""
    return bhalf_apply(adjoint_sweep(spec, traj, spec.rinv * d), taps)


def gamma(b):
    """Gamma = [b_1 - b_0, ..., b_L - b_0] (Eq. (Gamma)); shape (n, L)."""
    return (b[1:] - b[0]).T.copy()


def apply_A(spec, traj, V, taps):
    """A v = U_B^T G^T R^{-1} G U_B v for each row of V on its own trajectory.

    ``traj``: (M, N+1, n) with one trajectory per row of V.
    """
    u = bhalf_apply(V, taps)
    gv = tangent_sweep(spec, traj, u)
    return bhalf_apply(adjoint_sweep(spec, traj, spec.rinv * gv), taps)


def hvp(spec, traj, V, taps, identity=True):
    """(I + A) v (or A v) row by row."""
    av = apply_A(spec, traj, V, taps)
    return V + av if identity else av


def dense_A(spec, traj1, taps):
    """A assembled column by column for one trajectory (small n only)."""
    n = spec.n
    E = np.eye(n)
    tr = np.broadcast_to(traj1[None], (n,) + traj1.shape)
    return apply_A(spec, tr, E, taps).T


def cost_J(Hx, x, b):
    """Quadratic cost J(dz) = 1/2 dz^T H dz - b^T dz (up to a constant)."""
    return 0.5 * np.sum(x * Hx, -1) - np.sum(b * x, -1)


# ---------------------------------------------------------------------------
# q-pass Nystrom approximation (Section 3.2.3, Algorithm 1; Appendix B shift)
# ---------------------------------------------------------------------------


def nystrom(apply_a, Phi, k, q=1, shift_eps=np.finfo(np.float64).eps, evd_rtol=1e-12):
    """Algorithm 1.  ``apply_a`` maps an (n, ell) block to A times it.

    Returns (S_k (n, k), D_k (k,), info) with D_k descending.

    The small matrix W = Phi^T A Phi is inverted through its Cholesky factor
    (Algorithm 1).  If that breaks down, the algorithm is rerun on the
    shifted matrix A + nu I with nu = eps ||A Phi||_F and nu is subtracted
    from the eigenvalues (Appendix B, shift).  If the shifted factorisation
    also breaks down -- Phi itself numerically rank deficient, e.g. when B
    has few non-negligible eigenvalues -- W is inverted by a truncated
    eigendecomposition (Appendix B, third variant): W^+ = V diag(1/mu) V^T
    over the eigenvalues mu > evd_rtol * max(mu), T = R_Y V diag(mu^{-1/2}).
    The approximation then has rank r at most the number of kept mu, and
    only its modes with D > evd_rtol * max(D) carry information, so
    k_eff = min(k, their count): columns k_eff..k-1 of S_k and the matching
    entries of D_k are returned as zeros (the LMP acts as the identity
    there).  ``info['path']`` is 'cholesky', 'shift' or 'evd' and
    ``info['rank']`` is k_eff (k on the first two paths).
    """
    Phi = np.asarray(Phi, dtype=np.float64)
    Y = apply_a(Phi)
    Q, R = np.linalg.qr(Y)
    for _ in range(2, q + 1):
        Phi = Q
        Y = apply_a(Phi)
        Q, R = np.linalg.qr(Y)
    nu = 0.0
    path = "cholesky"
    W = Phi.T @ Y
    W = 0.5 * (W + W.T)
    try:
        L = np.linalg.cholesky(W)
        T = np.linalg.solve(L, R.T).T           # T = R_Y C^{-1}, C = L^T (W = C^T C)
    except np.linalg.LinAlgError:
        nu = shift_eps * np.linalg.norm(Y)
        Ys = Y + nu * Phi
        Qs, Rs = np.linalg.qr(Ys)
        Ws = Phi.T @ Ys
        Ws = 0.5 * (Ws + Ws.T)
        try:
            L = np.linalg.cholesky(Ws)
            Y, Q, R = Ys, Qs, Rs
            T = np.linalg.solve(L, R.T).T
            path = "shift"
        except np.linalg.LinAlgError:
            nu = 0.0
            path = "evd"
            mu, V = np.linalg.eigh(W)
            keep = mu > evd_rtol * max(mu.max(), 0.0)
            f = np.zeros_like(mu)
            f[keep] = 1.0 / np.sqrt(mu[keep])
            T = R @ (V * f)                       # T T^T = R_Y W^+ R_Y^T
    U, s, _ = np.linalg.svd(T)
    S = Q @ U
    D = s * s - nu
    D = np.maximum(D, 0.0)
    S, D = S[:, :k].copy(), D[:k].copy()
    rank = k
    if path == "evd":
        rank = min(k, int(keep.sum()), int(np.sum(D > evd_rtol * max(D.max(), 0.0))))
        S[:, rank:] = 0.0
        D[rank:] = 0.0
    return S, D, {"shift": nu, "path": path, "Y": Y, "Q": Q, "R": R, "rank": rank}


# ---------------------------------------------------------------------------
# Scaled spectral LMP (Section 3.1)
# ---------------------------------------------------------------------------


def theta_value(mode, D, theta_given=1.0):
    """theta: given, lambda_k(I+A), or (lambda_k(I+A) + lambda_n(I+A))/2 with
    lambda_n(I+A) = 1 (Section 3.1).  ``D`` holds the retained modes only
    (an empty D, a sketch without information, gives lambda_k = 1)."""
    if mode == 0:
        return float(theta_given)
    lam_k = 1.0 + (float(D[-1]) if len(D) else 0.0)
    if mode == 1:
        return lam_k
    return 0.5 * (lam_k + 1.0)


def lmp_coeffs(D, theta):
    """c_i = theta / (1 + lambda_i(A)) - 1 on the diagonal of P_theta - I."""
    return theta / (1.0 + D) - 1.0


def lmp_apply(S, c, R):
    """P_theta r = r + S_k diag(c) S_k^T r for each row r of R."""
    return R + ((R @ S) * c) @ S.T


def lmp_dense(S, c):
    return np.eye(S.shape[0]) + (S * c) @ S.T


def lmp_split_coeffs(D, theta):
    """s_i = sqrt(theta) (1 + lambda_i(A))^{-1/2} - 1: the factor
    U_theta = U_theta^T = I + S_k diag(s) S_k^T of P_theta = U_theta U_theta^T
    (Section 3.1, Eq. (lmp))."""
    return np.sqrt(theta) / np.sqrt(1.0 + D) - 1.0


# ---------------------------------------------------------------------------
# Preconditioned CG (Section 2.3), all members at once
# ---------------------------------------------------------------------------

CONVERGED, MAXIT, NAN, BREAKDOWN = 0, 1, 2, 3


def pcg(apply_h, b, precond=None, tol=1e-6, maxit=100, x0=None, fixed_iters=None):
    """Standard PCG on H x = b for every row of b.

    Stops a row when ||r_i|| / ||b|| <= tol on the recurrence residual (or,
    with ``fixed_iters`` (an int or one count per row), after exactly that
    many iterations).
    Returns dict(x, iters, relres, status, J) where J[i] lists the quadratic
    cost at each iterate (Eq. (quadratic cost) in the control variable).
    """
    b = np.asarray(b, dtype=np.float64)
    M, n = b.shape
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_h(x) if x0 is not None else b.copy()
    bnorm = np.linalg.norm(b, axis=1)
    P = (lambda v: v) if precond is None else precond
    z = P(r)
    p = z.copy()
    rz = np.sum(r * z, 1)
    iters = np.zeros(M, dtype=np.int64)
    status = np.full(M, MAXIT, dtype=np.int64)
    relres = np.where(bnorm > 0, np.linalg.norm(r, axis=1) / np.where(bnorm > 0, bnorm, 1), 0.0)
    active = np.ones(M, dtype=bool)
    if fixed_iters is not None:
        fixed = np.broadcast_to(np.asarray(fixed_iters, dtype=np.int64), (M,))
        limit = int(fixed.max()) if M else 0
        active &= fixed > 0
    else:
        limit = maxit
    if fixed_iters is None:
        done = relres <= tol
        status[done] = CONVERGED
        active &= ~done
    Jhist = [[0.5 * float(np.dot(x[m], b[m] - r[m])) - float(np.dot(b[m], x[m]))]
             for m in range(M)]
    for it in range(1, limit + 1):
        if fixed_iters is not None:
            active &= fixed >= it
        if not active.any():
            break
        q = apply_h(p)
        pq = np.sum(p * q, 1)
        bad = active & ~(pq > 0)
        status[bad] = BREAKDOWN
        active &= ~bad
        alpha = np.where(active, rz / np.where(active, pq, 1.0), 0.0)
        x = x + alpha[:, None] * p
        r = r - alpha[:, None] * q
        rr = np.linalg.norm(r, axis=1)
        relres = np.where(active, rr / np.where(bnorm > 0, bnorm, 1.0), relres)
        iters = np.where(active, it, iters)
        for m in np.nonzero(active)[0]:
            # J(x) = 1/2 x^T H x - b^T x with H x = b - r
            Jhist[m].append(0.5 * float(np.dot(x[m], b[m] - r[m])) - float(np.dot(b[m], x[m])))
        nanrow = active & ~np.isfinite(rr)
        status[nanrow] = NAN
        active &= ~nanrow
        if fixed_iters is None:
            done = active & (relres <= tol)
            status[done] = CONVERGED
            active &= ~done
        else:
            active &= fixed > it
        if not active.any():
            break
        z = P(r)
        rz_new = np.sum(r * z, 1)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        rz = np.where(active, rz_new, rz)
        p = np.where(active[:, None], z + beta[:, None] * p, p)
    if fixed_iters is not None:
        status[:] = np.where(status == BREAKDOWN, BREAKDOWN, CONVERGED)
    return {"x": x, "iters": iters, "relres": relres, "status": status, "J": Jhist}


def lanczos_cg(apply_h, b, iters):
    """Ritz pairs of H from conjugate gradients (Section 3: spectral LMPs
    built from the Ritz pairs of an earlier CG run; the CG-Lanczos relation).

    CG without preconditioner from x0 = 0 on H x = b (b one vector) for
    ``iters`` iterations.  Its residuals, normalised with alternating signs,
    v_j = (-1)^j r_j / |r_j|, are the Lanczos basis V of the Krylov space
    K_iters(H, b), and its coefficients give the tridiagonal T = V^T H V:
      T[j, j]   = 1/alpha_j + beta_{j-1}/alpha_{j-1}   (no second term at j = 0)
      T[j, j+1] = sqrt(beta_j) / alpha_j
    with alpha_j = |r_j|^2 / p_j^T H p_j and beta_j = |r_{j+1}|^2 / |r_j|^2.
    The eigenpairs (theta_i, y_i) of T give the Ritz pairs (theta_i, V y_i).
    Returns dict(V [n x iters], T, alpha, beta, theta (descending), S = the
    Ritz vectors [n x iters] in the same order, eta = T's next off-diagonal
    sqrt(beta_{iters-1}) / alpha_{iters-1}: |H s_i - theta_i s_i| = eta |y_i[-1]|)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.shape[0]
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    V = np.zeros((n, iters))
    alpha = np.zeros(iters)
    beta = np.zeros(iters)
    for j in range(iters):
        V[:, j] = (-1.0) ** j * r / np.sqrt(rr)
        q = np.asarray(apply_h(p[None, :]), dtype=np.float64).ravel()
        alpha[j] = rr / float(p @ q)
        r = r - alpha[j] * q
        rr_new = float(r @ r)
        beta[j] = rr_new / rr
        p = r + beta[j] * p
        rr = rr_new
    T = np.zeros((iters, iters))
    for j in range(iters):
        T[j, j] = 1.0 / alpha[j] + (beta[j - 1] / alpha[j - 1] if j > 0 else 0.0)
        if j + 1 < iters:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(beta[j]) / alpha[j]
    theta, Y = np.linalg.eigh(T)
    order = np.argsort(theta)[::-1]
    theta, Y = theta[order], Y[:, order]
    return {"V": V, "T": T, "alpha": alpha, "beta": beta, "theta": theta, "S": V @ Y, "Y": Y,
            "eta": np.sqrt(beta[-1]) / alpha[-1]}


def pcg_split(apply_h, b, S, s, tol=1e-6, maxit=100, fixed_iters=None):
    """CG on the split-preconditioned system U H U y = U b, x = U y, with the
    symmetric factor U = I + S diag(s) S^T of P = U U^T (Section 3.1, Eq.
    (lmp)).  In exact arithmetic x_i equals the i-th iterate of pcg with P.
    The stopping test is CG's own: ||U (b - H x_i)|| / ||U b|| <= tol.
    Returns pcg's dict with x mapped back (J is the same cost: 1/2 y^T U H U y
    - (U b)^T y = J(U y))."""
    U = lambda R: lmp_apply(S, s, R)
    res = pcg(lambda V: U(apply_h(U(V))), U(np.asarray(b, dtype=np.float64)), None, tol=tol, maxit=maxit,
              fixed_iters=fixed_iters)
    res["y"] = res["x"]
    res["x"] = U(res["y"])
    return res


# ---------------------------------------------------------------------------
# The whole path for one problem
# ---------------------------------------------------------------------------


def eda_pipeline(spec, xb, y, taps, tol=1e-6, maxit=500, use_lmp=True, fixed_iters=None,
                 phi=None, q=1, x0=None):
    """Setup, RHS, Gamma sketch of the control Hessian, Nystrom, LMP and PCG."""
    traj = member_trajectories(spec, xb)
    d = innovations(spec, traj, y)
    b = rhs(spec, traj, d, taps)
    out = {"traj": traj, "d": d, "b": b}
    ctrl = traj[0:1]
    if use_lmp:
        Phi = gamma(b)[:, : spec.ell] if phi is None else phi

        def apply_ctrl(block):
            tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
            return apply_A(spec, tr, block.T.copy(), taps).T

        S, D, info = nystrom(apply_ctrl, Phi, spec.k, q=q)
        r = info["rank"]
        theta = theta_value(spec.theta_mode, D[:r], spec.theta)
        c = lmp_coeffs(D, theta)
        c[r:] = 0.0
        out.update(S=S, D=D, theta=theta, c=c, shift=info["shift"], Y=info["Y"])
        P = lambda R: lmp_apply(S, c, R)
    else:
        P = None
    res = pcg(lambda V: hvp(spec, traj, V, taps), b, P, tol=tol, maxit=maxit,
              fixed_iters=fixed_iters, x0=x0)
    out.update(res)
    return out
