"""Pins of the oracle's Hessian, Nystrom approximation, LMP and PCG
(Section 2.3 system with CVT; Section 3.1 LMP; Section 3.2.2 Gamma;
Section 3.2.3 Algorithm 1) against closed forms, finite differences,
library routines on tiny inputs and invariants."""
import numpy as np
import pytest

import eda_synth as S
import oracle as O


def tiny_problem(seed=0, n=40, N=20, members=11, every_step=4, L=2.0, spinup=1000):
    steps, ptr, idx = S.regular_obs(n, N, 2, every_step)
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=1.0,
                  sigma_b=1.0, length_scale=L, n_members=members, ell=members - 1,
                  k=members - 1, seed=seed, spinup=spinup)
    taps = O.bhalf_taps(n, L, 1.0)
    dr = S.draws(spec)
    xt0, xb, y = O.twin(spec, dr, taps)
    traj = O.member_trajectories(spec, xb)
    return spec, taps, xb, y, traj


def test_hessian_matches_finite_differences_of_nonlinear_model():
    spec, taps, xb, y, traj = tiny_problem(n=16, N=8, members=2, every_step=2)
    n = spec.n
    # G_fd: central differences of x0 -> [H_t x_t]_t through the NONLINEAR model
    eps = 1e-5

    def gen_obs(x0):
        return O.obs_gather(spec, O.trajectory(x0, spec.F, spec.dt, spec.nsteps))

    G = np.stack([(gen_obs(xb[0] + eps * e) - gen_obs(xb[0] - eps * e)) / (2 * eps)
                  for e in np.eye(n)], axis=1)
    U = O.bhalf_dense(n, taps)
    A_fd = U.T @ G.T @ np.diag(spec.rinv) @ G @ U
    A = O.dense_A(spec, traj[0], taps)
    assert np.linalg.norm(A - A_fd) <= 1e-7 * np.linalg.norm(A)


def rk4_amplification(z):
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


@pytest.mark.parametrize("n,L,every", [(24, 2.0, 3), (40, 3.0, 5)])
def test_hessian_circulant_closed_form_at_fixed_point(n, L, every):
    # At x = F 1 the step propagator is R(dt J), J = F (S_{+1} - S_{-2}) - I circulant;
    # with H_t = I at every obs step, A is circulant with eigenvalues
    # b_m sum_t |R(dt mu_m)|^{2t} / sigma_o^2.
    N = 12
    steps = np.arange(every, N + 1, every, dtype=np.int32)
    ptr = (np.arange(len(steps) + 1) * n).astype(np.int32)
    idx = np.tile(np.arange(n, dtype=np.int32), len(steps))
    sig_o = 0.7
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=sig_o,
                  sigma_b=1.1, length_scale=L, n_members=1, ell=1, k=1)
    taps = O.bhalf_taps(n, L, 1.1)
    traj = O.trajectory(np.full(n, spec.F), spec.F, spec.dt, N)
    A = O.dense_A(spec, traj, taps)
    th = 2 * np.pi * np.arange(n) / n
    mu = spec.F * (np.exp(1j * th) - np.exp(-2j * th)) - 1
    beta = taps[0] + 2 * sum(taps[d] * np.cos(th * d) for d in range(1, len(taps)))
    amp = np.abs(rk4_amplification(spec.dt * mu)) ** 2
    closed = beta ** 2 * sum(amp ** int(t) for t in steps) / sig_o ** 2
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    np.testing.assert_allclose(np.sort(ev), np.sort(closed), rtol=1e-10,
                               atol=1e-12 * closed.max())


def test_hessian_spd_and_unit_cluster():
    spec, taps, xb, y, traj = tiny_problem()
    A = O.dense_A(spec, traj[0], taps)
    assert np.linalg.norm(A - A.T) <= 1e-12 * np.linalg.norm(A)
    H = np.eye(spec.n) + A
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev.min() >= 1 - 1e-10
    # <H u, v> = <u, H v> through the matrix-free product
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((2, spec.n))
    Hu = O.hvp(spec, traj[:1], u[None], taps)[0]
    Hv = O.hvp(spec, traj[:1], v[None], taps)[0]
    assert abs(Hu @ v - u @ Hv) <= 1e-12 * abs(Hu @ v)


def test_unit_eigenvalue_multiplicity_with_few_obs():
    # obs of 10 variables at one step: rank(A) <= p = 10, so I + A has at
    # least n - p eigenvalues exactly 1 (Section 2.3).
    n, N = 40, 10
    steps = np.array([N], dtype=np.int32)
    idx = np.arange(0, n, 4, dtype=np.int32)
    ptr = np.array([0, len(idx)], dtype=np.int32)
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=1.0,
                  sigma_b=1.0, length_scale=2.0, n_members=1, ell=1, k=1)
    taps = O.bhalf_taps(n, 2.0, 1.0)
    rng = np.random.default_rng(5)
    traj = O.trajectory(O.trajectory(spec.F + rng.standard_normal(n), spec.F, spec.dt, 500)[-1],
                        spec.F, spec.dt, N)
    H = np.eye(n) + O.dense_A(spec, traj, taps)
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert np.sum(np.abs(ev - 1) < 1e-10) >= n - len(idx)


def test_pcg_matches_dense_solve():
    spec, taps, xb, y, traj = tiny_problem()
    d = O.innovations(spec, traj, y)
    b = O.rhs(spec, traj, d, taps)
    ref = np.stack([np.linalg.solve(np.eye(spec.n) + O.dense_A(spec, traj[m], taps), b[m])
                    for m in range(spec.n_members)])
    res = O.pcg(lambda V: O.hvp(spec, traj, V, taps), b, tol=1e-13, maxit=200)
    err = np.linalg.norm(res["x"] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-10
    assert (res["status"] == O.CONVERGED).all()
    # a-priori bound: lambda_min(H) >= 1 so ||x - x*|| <= ||b - H x||
    res6 = O.pcg(lambda V: O.hvp(spec, traj, V, taps), b, tol=1e-6, maxit=200)
    true_r = b - O.hvp(spec, traj, res6["x"], taps)
    assert (np.linalg.norm(res6["x"] - ref, axis=1)
            <= np.linalg.norm(true_r, axis=1) * (1 + 1e-9)).all()


def nonlinear_cost(spec, taps, xb0, y0, dz):
    """Eq. (1) in the control variable (Section 2.3, CVT dx = U_B dz):
    1/2 ||dz||^2 + 1/2 sum_t ||y_t - H_t M_{0->t}(x_b + U_B dz)||^2_{R^-1},
    through the NONLINEAR model (no tangent linear, no adjoint)."""
    x0 = xb0 + O.bhalf_apply(dz, taps)
    dep = y0 - O.obs_gather(spec, O.trajectory(x0, spec.F, spec.dt, spec.nsteps))
    return 0.5 * float(dz @ dz) + 0.5 * float(np.sum(spec.rinv * dep * dep))


def test_rhs_is_minus_the_gradient_of_the_nonlinear_cost():
    # b = U_B^T G^T R^{-1} d is minus the gradient of the cost at dz = 0
    # (Section 2.3: the first Gauss-Newton step solves (I + A) dz = b).
    # Central differences of the nonlinear cost catch a sign, a missing
    # R^{-1} or U_B, or a wrong observation time in rhs(); sigma_o and
    # sigma_b differ from 1 so that R^{-1} and the U_B scale are visible.
    n, N = 32, 12
    steps, ptr, idx = S.regular_obs(n, N, 3, 4)
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=0.5,
                  sigma_b=0.8, length_scale=2.5, n_members=2, ell=1, k=1, spinup=500)
    taps = O.bhalf_taps(n, 2.5, 0.8)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    eps = 1e-4
    for m in range(2):
        g = np.array([(nonlinear_cost(spec, taps, xb[m], y[m], eps * e)
                       - nonlinear_cost(spec, taps, xb[m], y[m], -eps * e)) / (2 * eps) for e in np.eye(n)])
        assert np.linalg.norm(g + b[m]) <= 1e-6 * np.linalg.norm(b[m])


def test_pcg_from_an_initial_guess():
    # the x0 branch of pcg: r_0 = b - H x0, converged to the dense solution,
    # and CG from x0 on H x = b takes the same steps as CG from 0 on
    # H e = b - H x0 (Section 2.3; x = x0 + e)
    spec, taps, xb, y, traj = tiny_problem(seed=7)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    Hd = [np.eye(spec.n) + O.dense_A(spec, traj[m], taps) for m in range(spec.n_members)]
    ref = np.stack([np.linalg.solve(Hd[m], b[m]) for m in range(spec.n_members)])
    x0 = np.random.default_rng(4).standard_normal(b.shape) * np.linalg.norm(ref, axis=1, keepdims=True) \
        / np.sqrt(spec.n)
    hv = lambda V: O.hvp(spec, traj, V, taps)
    res = O.pcg(hv, b, tol=1e-13, maxit=300, x0=x0)
    assert (np.linalg.norm(res["x"] - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() <= 1e-10
    # the same r_0 = b - H x0 both ways (CG amplifies a 1e-16 difference in
    # it), so only the accumulation of x differs; and r_0 itself against
    # the dense operator
    r0 = b - hv(x0)
    r0d = np.stack([b[m] - Hd[m] @ x0[m] for m in range(spec.n_members)])
    assert np.abs(r0 - r0d).max() <= 1e-12 * np.abs(r0d).max()
    for K in (1, 4, 9):
        a = O.pcg(hv, b, tol=0, maxit=K, x0=x0, fixed_iters=K)["x"]
        e = O.pcg(hv, r0, tol=0, maxit=K, fixed_iters=K)["x"]
        assert (np.linalg.norm(a - (x0 + e), axis=1) / np.linalg.norm(a, axis=1)).max() <= 1e-12


def test_cost_and_its_history_along_pcg():
    # J(x) = 1/2 x^T H x - b^T x: J(x) - J(x*) = 1/2 (x - x*)^T H (x - x*) for
    # any x (x* = H^{-1} b), and CG minimises J over nested Krylov spaces, so
    # the history pcg records never increases and ends at J(x_K)
    spec, taps, xb, y, traj = tiny_problem(seed=8)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    H = np.eye(spec.n) + O.dense_A(spec, traj[0], taps)
    H = 0.5 * (H + H.T)
    xs = np.linalg.solve(H, b[0])
    rng = np.random.default_rng(2)
    for _ in range(3):
        x = xs + rng.standard_normal(spec.n)
        e = x - xs
        lhs = O.cost_J(H @ x, x, b[0]) - O.cost_J(H @ xs, xs, b[0])
        assert abs(lhs - 0.5 * e @ H @ e) <= 1e-10 * (0.5 * e @ H @ e)
    res = O.pcg(lambda V: O.hvp(spec, traj[:1], V, taps), b[:1], tol=0, maxit=25, fixed_iters=25)
    J = np.array(res["J"][0])
    assert len(J) == 26 and J[0] == 0.0
    assert (np.diff(J) <= 1e-12 * abs(J).max()).all()
    xk = res["x"][0]
    assert abs(J[-1] - O.cost_J(H @ xk, xk, b[0])) <= 1e-10 * abs(J[-1])
    assert J[-1] >= O.cost_J(H @ xs, xs, b[0]) - 1e-10 * abs(J[-1])


def test_pcg_with_lmp_matches_dense_solve():
    spec, taps, xb, y, traj = tiny_problem(seed=3)
    out = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=200)
    ref = np.stack([np.linalg.solve(np.eye(spec.n) + O.dense_A(spec, traj[m], taps), out["b"][m])
                    for m in range(spec.n_members)])
    err = np.linalg.norm(out["x"] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-10


def control_apply(spec, traj, taps):
    ctrl = traj[0:1]

    def f(block):
        tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
        return O.apply_A(spec, tr, block.T.copy(), taps).T
    return f


def test_nystrom_full_rank_recovers_eigenpairs():
    spec, taps, xb, y, traj = tiny_problem()
    A = O.dense_A(spec, traj[0], taps)
    A = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(A)
    lam, V = lam[::-1], V[:, ::-1]
    Phi = S.gaussian_matrix(spec.n, spec.n, 11)
    Sk, D, _ = O.nystrom(control_apply(spec, traj, taps), Phi, 10)
    np.testing.assert_allclose(D, lam[:10], rtol=1e-8)
    # eigenvectors, up to sign, for well-separated eigenvalues
    for i in range(10):
        gap = min(abs(lam[i] - lam[j]) for j in range(spec.n) if j != i)
        if gap > 1e-3 * lam[0]:
            assert abs(abs(Sk[:, i] @ V[:, i]) - 1) < 1e-8


def test_nystrom_exact_for_low_rank():
    # obs of p_t < n variables at one step: rank(A) <= p_t; a sketch with
    # ell = p_t generic columns spans range(A), so A_N = A (Section 3.2.3).
    n, N = 30, 6
    idx = np.arange(0, n, 3, dtype=np.int32)
    spec = S.Spec(n=n, nsteps=N, obs_steps=np.array([N], np.int32),
                  obs_ptr=np.array([0, len(idx)], np.int32), obs_idx=idx, sigma_o=1.0,
                  sigma_b=1.0, length_scale=2.0, n_members=1, ell=len(idx), k=len(idx))
    taps = O.bhalf_taps(n, 2.0, 1.0)
    rng = np.random.default_rng(8)
    traj = O.trajectory(O.trajectory(spec.F + rng.standard_normal(n), spec.F, spec.dt, 300)[-1],
                        spec.F, spec.dt, N)[None]
    A = O.dense_A(spec, traj[0], taps)
    Phi = S.gaussian_matrix(n, len(idx), 9)
    Sk, D, _ = O.nystrom(control_apply(spec, traj, taps), Phi, len(idx))
    AN = (Sk * D) @ Sk.T
    assert np.linalg.norm(AN - A) <= 1e-10 * np.linalg.norm(A)
    assert np.allclose(Sk.T @ Sk, np.eye(len(idx)), atol=1e-12)


def test_nystrom_invariant_under_column_mixing():
    spec, taps, xb, y, traj = tiny_problem()
    f = control_apply(spec, traj, taps)
    Phi = S.gaussian_matrix(spec.n, 10, 12)
    G = S.gaussian_matrix(10, 10, 13) + 3 * np.eye(10)
    S1, D1, _ = O.nystrom(f, Phi, 10)
    S2, D2, _ = O.nystrom(f, Phi @ G, 10)
    np.testing.assert_allclose(D1, D2, rtol=1e-9)
    np.testing.assert_allclose((S1 * D1) @ S1.T, (S2 * D2) @ S2.T, atol=1e-9 * D1[0])


def test_nystrom_power_pass_improves_top_eigenvalue():
    spec, taps, xb, y, traj = tiny_problem()
    A = O.dense_A(spec, traj[0], taps)
    lam = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))[::-1]
    f = control_apply(spec, traj, taps)
    Phi = S.gaussian_matrix(spec.n, 8, 14)
    _, D1, _ = O.nystrom(f, Phi, 4, q=1)
    _, D2, _ = O.nystrom(f, Phi, 4, q=2)
    e1 = np.abs(D1 - lam[:4]) / lam[:4]
    e2 = np.abs(D2 - lam[:4]) / lam[:4]
    assert e2.sum() <= e1.sum() + 1e-12
    # Nystrom never overestimates (A_N <= A in the Loewner order)
    assert (D1 <= lam[:4] * (1 + 1e-10)).all()


def test_nystrom_shift_fallback_on_rank_deficient_sketch():
    spec, taps, xb, y, traj = tiny_problem()
    f = control_apply(spec, traj, taps)
    Phi = S.gaussian_matrix(spec.n, 6, 15)
    Phi = np.concatenate([Phi, Phi[:, :2]], axis=1)   # two repeated columns
    Sk, D, info = O.nystrom(f, Phi, 4)
    assert info["shift"] > 0
    Sk0, D0, _ = O.nystrom(f, Phi[:, :6], 4)
    np.testing.assert_allclose(D, D0, rtol=1e-6)


@pytest.mark.parametrize("theta", [1.0, 2.5])
def test_lmp_with_exact_eigenpairs(theta):
    spec, taps, xb, y, traj = tiny_problem()
    A = O.dense_A(spec, traj[0], taps)
    A = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(A)
    lam, V = lam[::-1], V[:, ::-1]
    k = 6
    c = O.lmp_coeffs(lam[:k], theta)
    P = O.lmp_dense(V[:, :k], c)
    H = np.eye(spec.n) + A
    # P H on span(S_k) is theta; on the complement it is H itself (Section 3.1)
    PH = P @ H
    np.testing.assert_allclose(PH @ V[:, :k], theta * V[:, :k], atol=1e-10 * lam[0])
    np.testing.assert_allclose(PH @ V[:, k:], V[:, k:] * (1 + lam[k:]), atol=1e-10 * lam[0])
    # the symmetric split factor U_theta squares to P_theta
    Uf = np.eye(spec.n) + V[:, :k] @ np.diag(np.sqrt(theta / (1 + lam[:k])) - 1) @ V[:, :k].T
    np.testing.assert_allclose(Uf @ Uf.T, P, atol=1e-12)
    # matrix-free apply equals the dense operator
    R = np.random.default_rng(0).standard_normal((3, spec.n))
    np.testing.assert_allclose(O.lmp_apply(V[:, :k], c, R), R @ P.T, atol=1e-12)


def test_theta_choices():
    D = np.array([9.0, 5.0, 3.0])
    assert O.theta_value(0, D, 1.7) == 1.7
    assert O.theta_value(1, D) == 4.0
    assert O.theta_value(2, D) == 2.5


def test_gamma_covariance_is_A_plus_A2_on_linear_twin():
    # Linear twin: truth and backgrounds at the fixed point x = F 1 with tiny
    # error scales s (B = s^2 C, R = s^2 I), so the model acts linearly on the
    # perturbations; A and gamma_j are independent of s and
    # cov(gamma_j) = A + A^2 exactly (Section 3.2.2).
    n, N, s = 12, 6, 1e-7
    steps = np.array([3, 6], dtype=np.int32)
    idx1 = np.arange(0, n, 2, dtype=np.int32)
    idx = np.tile(idx1, 2)
    ptr = np.array([0, len(idx1), 2 * len(idx1)], dtype=np.int32)
    draws = 4000
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=s,
                  sigma_b=s, length_scale=1.5, n_members=draws + 1, ell=draws, k=1,
                  spinup=0, spin_sigma=0.0)
    taps = O.bhalf_taps(n, 1.5, s)
    dr = S.draws(spec, seed=21)
    xt0, xb, y = O.twin(spec, dr, taps)
    traj = O.member_trajectories(spec, xb)
    d = O.innovations(spec, traj, y)
    b = O.rhs(spec, traj, d, taps)
    G = O.gamma(b)
    cov = G @ G.T / draws
    A = O.dense_A(spec, traj[0], taps)
    target = A + A @ A
    rel = np.linalg.norm(cov - target) / np.linalg.norm(target)
    assert rel < 6.0 / np.sqrt(draws), rel
    # and the mean of gamma is zero to Monte-Carlo accuracy
    assert np.linalg.norm(G.mean(1)) < 6.0 * np.sqrt(np.trace(target) / draws)


def test_nystrom_truncated_evd_when_the_sketch_is_rank_deficient():
    # B with a length scale comparable to n has only a few non-negligible
    # eigenvalues, so Gamma (in the range of U_B) is numerically rank
    # deficient and no shift of A makes Phi^T A Phi definite; the truncated
    # eigendecomposition variant (Appendix B) still returns the Nystrom
    # approximation, which is exact on the span of the sketch:
    # S D S^T = A Phi (Phi^T A Phi)^+ Phi^T A.
    n, N = 41, 10
    steps, ptr, idx = S.regular_obs(n, N, 3, 2)
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=1.0,
                  sigma_b=1.0, length_scale=7.6, n_members=33, ell=32, k=31, spinup=300)
    taps = O.bhalf_taps(n, 7.6, 1.0)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    Phi = O.gamma(b)[:, :32]
    sv = np.linalg.svd(Phi, compute_uv=False)
    assert sv[-1] < 1e-6 * sv[0]          # numerically rank deficient
    f = control_apply(spec, traj, taps)
    Sk, D, info = O.nystrom(f, Phi, 31, evd_rtol=1e-12)
    assert info["path"] == "evd"
    A = O.dense_A(spec, traj[0], taps)
    Y = A @ Phi
    W = Phi.T @ Y
    mu, V = np.linalg.eigh(0.5 * (W + W.T))
    keep = mu > 1e-12 * mu.max()
    # rank r of the approximation < k: the first r columns are orthonormal
    # eigenvectors, the remaining ones (and their D) are zero.  Reading of
    # Appendix B (truncated eigendecomposition): A_N = Y W^+ Y^T has rank at
    # most the number of kept eigenvalues of W, and of its nonzero
    # eigenvalues only those above the truncation level carry information,
    # so r can fall below keep.sum() when Y maps kept directions to
    # negligible ones; hence r <= keep.sum(), not equality
    r = info["rank"]
    assert r <= keep.sum() < 31 and D[r - 1] > 1e-12 * D[0]
    np.testing.assert_allclose(Sk[:, :r].T @ Sk[:, :r], np.eye(r), atol=1e-12)
    assert not Sk[:, r:].any() and not D[r:].any()
    AN = Y @ (V[:, keep] / mu[keep]) @ V[:, keep].T @ Y.T
    np.testing.assert_allclose((Sk * D) @ Sk.T, AN, atol=1e-8 * np.abs(AN).max())
    # and A_N <= A: no eigenvalue exceeds A's
    lamA = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))[::-1]
    assert (D <= lamA[: len(D)] * (1 + 1e-8) + 1e-10 * lamA[0]).all()


def test_split_preconditioner_factor_and_iterates():
    # Section 3.1, Eq. (lmp): U_theta = U_theta^T with U U = P_theta, and CG
    # on U H U y = U b gives x = U y equal to the PCG iterates with P_theta
    # (U K_i(U H U, U b) = K_i(P H, P b), and the U H U-norm of y - y* is the
    # H-norm of x - x*), so both minimise the same error on the same space
    spec, taps, xb, y, traj = tiny_problem(seed=9)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    f = control_apply(spec, traj, taps)
    Sk, D, _ = O.nystrom(f, O.gamma(b)[:, : spec.ell], spec.k)
    for mode in (0, 1, 2):
        theta = O.theta_value(mode, D, 2.5)
        c = O.lmp_coeffs(D, theta)
        s = O.lmp_split_coeffs(D, theta)
        U = O.lmp_dense(Sk, s)
        Pm = O.lmp_dense(Sk, c)
        assert np.abs(U - U.T).max() <= 1e-14
        assert np.abs(U @ U - Pm).max() <= 1e-12 * np.abs(Pm).max()
        hv = lambda V: O.hvp(spec, traj, V, taps)
        for K in (1, 3, 6):
            a = O.pcg(hv, b, lambda R: O.lmp_apply(Sk, c, R), tol=0, maxit=K, fixed_iters=K)
            bsp = O.pcg_split(hv, b, Sk, s, tol=0, maxit=K, fixed_iters=K)
            err = np.linalg.norm(bsp["x"] - a["x"], axis=1) / np.linalg.norm(a["x"], axis=1)
            assert err.max() <= 1e-9, (mode, K, err.max())
            np.testing.assert_allclose(np.array(bsp["J"]), np.array(a["J"]), rtol=1e-9, atol=1e-12)
    ref = np.stack([np.linalg.solve(np.eye(spec.n) + O.dense_A(spec, traj[m], taps), b[m])
                    for m in range(spec.n_members)])
    res = O.pcg_split(hv, b, Sk, s, tol=1e-13, maxit=300)
    assert (np.linalg.norm(res["x"] - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() <= 1e-10


def test_lanczos_cg_relations_and_ritz_pairs():
    # Ritz pairs from CG (Section 3: spectral LMPs from the Ritz pairs of an
    # earlier CG run), pinned on an explicit SPD matrix with eigenvalues >= 1
    # (the spectrum class of I + A): the alternating-sign normalised
    # residuals are orthonormal, V^T H V is CG's tridiagonal, with as many
    # iterations as unknowns the Ritz values are the eigenvalues, and every
    # Ritz pair satisfies the Lanczos residual identity
    rng = np.random.default_rng(12)
    n = 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = 1.0 + np.geomspace(1e2, 1e-2, n)
    H = (Q * lam) @ Q.T
    b = rng.standard_normal(n)
    apply_h = lambda X: X @ H.T
    k = 6
    L = O.lanczos_cg(apply_h, b, k)
    V, T = L["V"], L["T"]
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(V.T @ H @ V, T, rtol=0, atol=1e-10 * np.abs(T).max())
    for i in range(k):
        s, th = L["S"][:, i], L["theta"][i]
        res = np.linalg.norm(H @ s - th * s)
        assert abs(res - L["eta"] * abs(L["Y"][-1, i])) <= 1e-9 * lam.max()
    assert (np.diff(L["theta"]) <= 0).all() and L["theta"][-1] >= 1.0 - 1e-12
    # as many iterations as unknowns, on a well-conditioned H (so that the
    # finite-precision Lanczos basis stays orthogonal): the Ritz values are
    # the eigenvalues and the Ritz vectors the eigenvectors (up to sign)
    m = 8
    Q2, _ = np.linalg.qr(rng.standard_normal((m, m)))
    lam2 = 1.0 + np.linspace(4.0, 0.1, m)
    H2 = (Q2 * lam2) @ Q2.T
    full = O.lanczos_cg(lambda X: X @ H2.T, rng.standard_normal(m), m)
    np.testing.assert_allclose(full["theta"], np.sort(lam2)[::-1], rtol=1e-9)
    for i in range(m):
        v = Q2[:, np.argsort(lam2)[::-1][i]]
        assert abs(abs(full["S"][:, i] @ v) - 1.0) < 1e-8


def test_lanczos_cg_on_the_control_hessian():
    # the same relations through the oracle's Hessian products of the tiny
    # EDA problem's control member (batch interface of hvp)
    spec = S.spec_tiny(seed=3)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    Hd = np.eye(spec.n) + O.dense_A(spec, traj[0], taps)
    L = O.lanczos_cg(lambda X: O.hvp(spec, traj[0:1], X, taps), b[0], 8)
    np.testing.assert_allclose(L["V"].T @ L["V"], np.eye(8), atol=1e-10)
    np.testing.assert_allclose(L["V"].T @ Hd @ L["V"], L["T"], rtol=0, atol=1e-9 * np.abs(L["T"]).max())
    ev = np.linalg.eigvalsh(Hd)
    assert L["theta"][0] <= ev[-1] * (1 + 1e-12) and L["theta"][-1] >= ev[0] * (1 - 1e-12)
    # the largest Ritz value converges first: within 1e-3 of lambda_max
    assert abs(L["theta"][0] - ev[-1]) <= 1e-3 * ev[-1]
