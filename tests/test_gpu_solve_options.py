"""eda_solve options against the FP64 oracle, through the C ABI: the cost
record J(x_i) along PCG (Section 2, Eq. (2); the paper's convergence plots),
the three choices of theta of the scaled spectral LMP (Section 3.1), and the
certified error stop ||r|| / (||x|| - ||r||) <= err_tol, which bounds the
relative error because every eigenvalue of I + A is at least 1 (Section 2.3)."""
from dataclasses import replace

import numpy as np
import pytest

import eda_synth as S
import oracle as O
from helpers import problem, rowrel

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_23571_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_lmp(spec, taps, xb, y):
    ref = O.eda_pipeline(spec, xb, y, taps, tol=0, maxit=1, fixed_iters=1)
    return ref["traj"], ref["b"], ref["S"], ref["D"]


def oracle_fixed(spec, traj, b, taps, S_, D_, K, theta_mode, theta_given=1.0):
    c = O.lmp_coeffs(D_, O.theta_value(theta_mode, D_, theta_given))
    return O.pcg(lambda V: O.hvp(spec, traj, V, taps), b, lambda R: O.lmp_apply(S_, c, R),
                 tol=0, maxit=K, fixed_iters=K)


def calm_members(spec, traj, b, taps, S_, D_, K, theta_mode, theta_given=1.0):
    """Members whose K-iteration iterate moves by less than 1e-12 when b is
    perturbed by 1e-16: there two FP64 implementations agree to 1e-10."""
    a = oracle_fixed(spec, traj, b, taps, S_, D_, K, theta_mode, theta_given)["x"]
    bp = b * (1 + 1e-16 * np.random.default_rng(0).standard_normal(b.shape))
    c = oracle_fixed(spec, traj, bp, taps, S_, D_, K, theta_mode, theta_given)["x"]
    return rowrel(c, a) < 1e-12


@pytest.mark.parametrize("mode,theta", [(P.EDA_THETA_GIVEN, 1.0), (P.EDA_THETA_GIVEN, 3.5),
                                        (P.EDA_THETA_LAMBDA_K, 1.0), (P.EDA_THETA_MID, 1.0)],
                         ids=["theta=1", "theta=3.5", "theta=lambda_k", "theta=mid"])
def test_theta_modes_and_cost_record_match_the_oracle(mode, theta):
    # one preconditioner (the oracle's S and eigenvalues, eda_set_lmp) on both
    # sides: the handle's theta_mode turns them into the LMP coefficients
    spec = replace(S.spec_tiny(seed=11), theta_mode=mode, theta=theta)
    taps, xb, y = problem(spec)
    traj, b, S_, D_ = oracle_lmp(spec, taps, xb, y)
    K = 6
    ref = oracle_fixed(spec, traj, b, taps, S_, D_, K, mode, theta)
    calm = calm_members(spec, traj, b, taps, S_, D_, K, mode, theta)
    assert calm.sum() >= 3
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_set_lmp(np.ascontiguousarray(S_.T), 1 + D_)
        dz = np.zeros_like(b)
        cost = np.zeros((spec.n_members, K + 1))
        it = np.zeros(spec.n_members, np.int32)
        h.eda_solve(dz, tol=0.0, maxit=K, use_lmp=True, cost_out=cost, iters_out=it)
        assert (it == K).all()
        assert (rowrel(dz, ref["x"])[calm] < 1e-10).all()
        Jo = np.array([ref["J"][m] for m in range(spec.n_members)])
        scale = np.abs(Jo).max(axis=1)
        assert (np.abs(cost - Jo).max(axis=1)[calm] <= 1e-10 * scale[calm]).all()
        # J never increases along CG, on every member
        assert (np.diff(cost, axis=1) <= 1e-12 * scale[:, None]).all()
        # the library's own LMP with this theta_mode: same eigenvalues, and
        # the cost curve of the control member follows the oracle's closely
        h.eda_sketch()
        ev = np.zeros(spec.k)
        h.eda_build_lmp(ev)
        np.testing.assert_allclose(ev, 1 + D_, rtol=1e-9)
        cost2 = np.zeros_like(cost)
        h.eda_solve(dz, tol=0.0, maxit=K, use_lmp=True, cost_out=cost2)
        assert np.abs(cost2 - Jo).max() <= 1e-6 * np.abs(Jo).max()


def test_cost_record_from_an_initial_guess_and_early_stops():
    # J(x0) first; after a member's last iteration the record is NaN
    spec = S.spec_tiny(seed=12)
    taps, xb, y = problem(spec)
    traj, b, S_, D_ = oracle_lmp(spec, taps, xb, y)
    x0 = 0.01 * np.random.default_rng(1).standard_normal(b.shape)
    Hx0 = O.hvp(spec, traj, x0, taps)
    J0 = O.cost_J(Hx0, x0, b)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_set_lmp(np.ascontiguousarray(S_.T), 1 + D_)
        maxit = 60
        dz = np.zeros_like(b)
        cost = np.zeros((spec.n_members, maxit + 1))
        it = np.zeros(spec.n_members, np.int32)
        st = np.zeros(spec.n_members, np.int32)
        h.eda_solve(dz, tol=1e-6, maxit=maxit, x0=x0, cost_out=cost, iters_out=it, status_out=st)
    assert (st == P.EDA_CONVERGED).all() and (it < maxit).all()
    np.testing.assert_allclose(cost[:, 0], J0, rtol=1e-10, atol=1e-10 * np.abs(J0).max())
    for m in range(spec.n_members):
        assert np.isfinite(cost[m, : it[m] + 1]).all() and np.isnan(cost[m, it[m] + 1:]).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_certified_error_stop(precision):
    # err_tol bounds the true relative error: check it against the dense
    # direct solve of the oracle's operator (n = 97, several members)
    spec = S.spec_small(97, 13, 6, every_var=3, every_step=3, length_scale=3.0, seed=13)
    spec = replace(spec, ell=5, k=5)
    taps, xb, y = problem(spec)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    exact = np.stack([np.linalg.solve(np.eye(spec.n) + O.dense_A(spec, traj[m], taps), b[m])
                      for m in range(spec.n_members)])
    prec = P.EDA_FP64 if precision == "fp64" else P.EDA_MIXED
    with P.Handle.from_spec(spec, taps, precision=prec) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_sketch()
        h.eda_build_lmp()
        for etol in (1e-4, 1e-8):
            dz = np.zeros_like(b)
            eb = np.zeros(spec.n_members)
            rr = np.zeros(spec.n_members)
            st = np.zeros(spec.n_members, np.int32)
            h.eda_solve(dz, err_tol=etol, maxit=2000, err_bound_out=eb, relres_out=rr, status_out=st)
            err = rowrel(dz, exact)
            assert (st == P.EDA_CONVERGED).all()
            assert (eb <= etol).all(), (etol, eb)
            assert (err <= eb * (1 + 1e-6) + 1e-13).all(), (etol, err, eb)
        # the bound of a relative-residual stop is reported, and also holds
        h.eda_solve(dz, tol=1e-6, maxit=2000, err_bound_out=eb, status_out=st)
        assert (st == P.EDA_CONVERGED).all() and np.isfinite(eb).all()
        assert (rowrel(dz, exact) <= eb * (1 + 1e-6) + 1e-13).all()
