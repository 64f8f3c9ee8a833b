"""The spectral LMP from Ritz pairs of an earlier CG run (Section 3), through
eda_ritz_lmp, against the oracle's CG-Lanczos relation (lanczos_cg): the
Ritz values, the LMP's action, and the solve it preconditions."""
import numpy as np
import pytest

import eda_synth as S
import oracle as O
from helpers import problem

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_23571_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# member 0 after 8 iterations keeps an orthogonal basis (no Ritz pair has
# converged); member 3 after 14 has converged its leading pair (residual
# about 3e-11) and lost orthogonality to about 1e-4; member 2's Hessian from
# member 5's right-hand side, passed as host memory
@pytest.mark.parametrize("member,iters,b_from", [(0, 8, None), (3, 14, None), (2, 10, 5)])
def test_ritz_pairs_and_lmp_match_the_oracle(member, iters, b_from):
    spec = S.spec_small(400, 12, 9, every_var=2, every_step=2, length_scale=4.0, ell=8, k=8, seed=21)
    taps, xb, y = problem(spec)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    rhs = b[member if b_from is None else b_from]
    L = O.lanczos_cg(lambda X: O.hvp(spec, traj[member:member + 1], X, taps), rhs, iters)
    k = spec.k
    D = L["theta"][:k] - 1.0
    c = O.lmp_coeffs(D, O.theta_value(spec.theta_mode, D, spec.theta))
    R = np.random.default_rng(member).standard_normal((spec.n_members, spec.n))
    ref = O.lmp_apply(L["S"][:, :k], c, R)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(xb, y)
        theta = h.eda_ritz_lmp(member=member, iters=iters, b=None if b_from is None else np.ascontiguousarray(rhs))
        Z = np.zeros_like(R)
        h.eda_lmp_apply(R, Z, 0, 0)
        # the preconditioned solve converges, in fewer iterations than without it
        dz = np.zeros((spec.n_members, spec.n))
        it_p = np.zeros(spec.n_members, np.int32)
        it_0 = np.zeros(spec.n_members, np.int32)
        st = np.zeros(spec.n_members, np.int32)
        h.eda_solve_batch(1e-8, 2000, None, True, dz, it_p, None, st)
        assert (st == P.EDA_CONVERGED).all()
        h.eda_solve_batch(1e-8, 2000, None, False, dz, it_0, None, st)
    # Ritz values: the leading ones converge first and agree closely; all
    # agree to the rounding the recurrences amplify over the iterations
    np.testing.assert_allclose(theta[:k], L["theta"][:k], rtol=1e-8)
    np.testing.assert_allclose(theta, L["theta"], rtol=1e-6)
    assert (np.diff(theta) <= 0).all()
    # the LMP's correction S diag(c) S^T R, relative to its own size.  Once
    # a Ritz pair has converged the Lanczos basis loses orthogonality along
    # it, by an amount that rounding decides; two runs of the recurrence with
    # different summation orders then differ by about that loss, so the bar
    # is FP64 rounding plus a few times the oracle's own loss of orthogonality
    orth = np.abs(L["V"].T @ L["V"] - np.eye(iters)).max()
    err = (np.linalg.norm(Z - ref, axis=1) / np.linalg.norm(ref - R, axis=1)).max()
    assert err < 1e-9 + 4.0 * orth, (err, orth)
    assert it_p.sum() < it_0.sum()


def test_ritz_lmp_on_a_mixed_handle():
    # the CG runs on the FP64 sweeps of a mixed handle; the installed LMP is
    # applied in FP32 (its S and arithmetic), to 1e-5 of the correction
    spec = S.spec_small(400, 12, 9, every_var=2, every_step=2, length_scale=4.0, ell=8, k=8, seed=21)
    taps, xb, y = problem(spec)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    L = O.lanczos_cg(lambda X: O.hvp(spec, traj[0:1], X, taps), b[0], 8)
    D = L["theta"][:spec.k] - 1.0
    c = O.lmp_coeffs(D, O.theta_value(spec.theta_mode, D, spec.theta))
    R = np.random.default_rng(5).standard_normal((spec.n_members, spec.n))
    ref = O.lmp_apply(L["S"][:, :spec.k], c, R)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        theta = h.eda_ritz_lmp(member=0, iters=8)
        Z = np.zeros_like(R)
        h.eda_lmp_apply(R, Z, 0, 0)
    np.testing.assert_allclose(theta, L["theta"], rtol=1e-8)
    assert (np.linalg.norm(Z - ref, axis=1) / np.linalg.norm(ref - R, axis=1)).max() < 1e-5


def test_ritz_lmp_refusals():
    spec = S.spec_small(200, 8, 5, every_var=2, every_step=2, length_scale=3.0, ell=4, k=4, seed=22)
    taps, xb, y = problem(spec)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        with pytest.raises(P.EdaError):
            h.eda_ritz_lmp(member=0, iters=4)  # before eda_set_trajectory
        h.eda_set_trajectory(xb, y)
        with pytest.raises(P.EdaError):
            h.eda_ritz_lmp(member=spec.n_members, iters=4)  # no such member
        with pytest.raises(P.EdaError):
            h.eda_ritz_lmp(member=0, iters=3)  # fewer iterations than the LMP rank
        with pytest.raises(P.EdaError):
            h.eda_ritz_lmp(member=0, iters=4, b=np.zeros(spec.n))  # a zero right-hand side
        h.eda_ritz_lmp(member=0, iters=4)
        path, rank, _ = h.eda_lmp_info()
        assert rank == spec.k
