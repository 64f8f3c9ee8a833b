"""The paper's sketch comparison (Section 4, Fig. 3) on the oracle, at a
size the CPU finishes in seconds: Algorithm 1 on the control member's
Hessian with Omega = Psi, A Psi (q = 2), B Psi, U_B^T Psi and Gamma, and the
median relative error of the leading eigenvalues of I + A against those of
the dense operator (numpy's symmetric eigensolver).  The paper reports that
Gamma and A Psi approximate the largest eigenvalues best; the test checks
that ordering, and the synthetic inputs the study uses."""
import numpy as np

import eda_synth as S
import oracle as O


def _small_paper_like():
    # the paper's observation pattern (every 10th variable at steps 4, 7, 10;
    # sigma_o = 0.05, sigma_b = 0.8) on n = 300
    n, N = 300, 10
    steps = np.array([4, 7, 10], dtype=np.int32)
    idx1 = np.arange(0, n, 10, dtype=np.int32)
    return S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=(np.arange(4) * len(idx1)).astype(np.int32),
                  obs_idx=np.tile(idx1, 3), sigma_o=0.05, sigma_b=0.8, length_scale=6.0, n_members=21,
                  ell=20, k=20, spinup=300, name="l96_n300_w10_m21")


def test_paper_spec_and_ensemble_draws():
    spec = S.spec_paper()
    assert (spec.n, spec.nsteps, spec.p, spec.n_members, spec.ell, spec.k) == (1500, 10, 150, 21, 20, 20)
    assert list(spec.obs_steps) == [4, 7, 10]
    assert (np.diff(spec.obs_idx[:50]) == 30).all() and spec.sigma_o == 0.05 and spec.sigma_b == 0.8
    a = S.ensemble_draws(spec, 0, 1)
    b = S.ensemble_draws(spec, 0, 2)
    # one truth and control member, other ensemble perturbations
    np.testing.assert_array_equal(a.eta_spin, b.eta_spin)
    np.testing.assert_array_equal(a.eta_b[0], b.eta_b[0])
    np.testing.assert_array_equal(a.eta_o[0], b.eta_o[0])
    assert not np.allclose(a.eta_b[1:], b.eta_b[1:])
    assert a.eta_b.shape == (spec.n_members, spec.n) and a.eta_o.shape == (spec.n_members, spec.p)


def test_gamma_and_power_sketch_approximate_the_leading_eigenvalues_best():
    spec = _small_paper_like()
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, _ = O.twin(spec, S.ensemble_draws(spec, 0, 0), taps)
    ctrl = O.member_trajectories(spec, xb)[0:1]
    A = O.dense_A(spec, ctrl[0], taps)
    lam = 1.0 + np.linalg.eigvalsh(0.5 * (A + A.T))[::-1][: spec.ell]

    def apply_ctrl(block):
        tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
        return O.apply_A(spec, tr, block.T.copy(), taps).T

    errs = {v: [] for v in ("psi", "a_psi", "b_psi", "ubt_psi", "gamma")}
    for seed in range(10):
        _, xb, y = O.twin(spec, S.ensemble_draws(spec, 0, 1000 + seed), taps)
        traj = O.member_trajectories(spec, xb)
        b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
        psi = S.gaussian_matrix(spec.ell, spec.n, 2000 + seed).T
        ub = O.bhalf_apply(psi.T, taps).T
        phis = {"psi": (psi, 1), "a_psi": (psi, 2), "b_psi": (O.bhalf_apply(ub.T, taps).T, 1),
                "ubt_psi": (ub, 1), "gamma": (O.gamma(b)[:, : spec.ell], 1)}
        for v, (phi, q) in phis.items():
            _, D, _ = O.nystrom(apply_ctrl, phi, spec.k, q=q)
            errs[v].append(np.abs(lam - 1.0 - D) / lam)
    med = {v: np.median(np.array(e), axis=0)[:5] for v, e in errs.items()}
    for best in ("gamma", "a_psi"):
        for other in ("psi", "b_psi", "ubt_psi"):
            assert (med[best] < med[other]).all(), (best, other, med[best], med[other])
