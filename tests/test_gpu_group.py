"""Uneven batching (many independent EDA problems in batched launches, the
PCG iteration captured in a CUDA graph) against the FP64 oracle, problem by
problem."""
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


def small_uneven(count=6, seed=3):
    # uneven sizes, windows, member counts, densities and length scales
    specs = S.specs_uneven(count, seed=seed, n_range=(40, 700), w_range=(6, 24), m_range=(3, 9))
    for s_ in specs:
        s_.spinup = 300
    return specs


def test_group_hvp_sweep_and_solve_match_oracle_fp64():
    specs = small_uneven()
    probs = [problem(s_) for s_ in specs]
    hs = [P.Handle.from_spec(s_, taps, precision=P.EDA_FP64) for s_, (taps, _, _) in zip(specs, probs)]
    with P.Group(hs) as g:
        g.eda_group_set_trajectories([xb for _, xb, _ in probs], [y for _, _, y in probs])
        g.eda_group_sketch()
        g.eda_group_build_lmp()
        g.eda_group_autotune()
        T = g.total_members
        dz = [np.zeros((s_.n_members, s_.n)) for s_ in specs]
        it = np.zeros(T, np.int32)
        rr = np.zeros(T)
        st = np.zeros(T, np.int32)
        g.eda_group_solve(1e-10, 2000, True, dz, it, rr, st)
    for h in hs:
        h.close()
    assert (st == P.EDA_CONVERGED).all()
    assert (rr <= 1e-10).all()
    off = 0
    for s_, (taps, xb, y), z in zip(specs, probs, dz):
        # against the oracle's 1e-13 solution of every member: since
        # lambda_min(I + A) >= 1 the error is at most the residual,
        # ||e|| <= ||r|| = relres ||b|| (1e-10 here, with slack for the gap
        # between recurrence and true residual)
        traj = O.member_trajectories(s_, xb)
        b = O.rhs(s_, traj, O.innovations(s_, traj, y), taps)
        ref = O.pcg(lambda V: O.hvp(s_, traj, V, taps), b, tol=1e-13, maxit=5000)["x"]
        e = np.linalg.norm(z - ref, axis=1)
        assert (e <= 1.5e-10 * np.linalg.norm(b, axis=1) + 1e-13).all(), (s_.name, e)
        assert rowrel(z, ref).max() < 1e-6
        off += s_.n_members


def test_group_sketch_matches_oracle_and_single_handles():
    specs = small_uneven(4, seed=11)
    probs = [problem(s_) for s_ in specs]
    hs = [P.Handle.from_spec(s_, taps, precision=P.EDA_FP64) for s_, (taps, _, _) in zip(specs, probs)]
    with P.Group(hs) as g:
        g.eda_group_set_trajectories([xb for _, xb, _ in probs], [y for _, _, y in probs])
        g.eda_group_sketch()
        g.eda_group_build_lmp()
    for s_, (taps, xb, y), h in zip(specs, probs, hs):
        ref = O.eda_pipeline(s_, xb, y, taps, tol=0, maxit=1, fixed_iters=1)
        ev = np.zeros(s_.k)
        # the group left every handle with its sketch and LMP built
        h.eda_build_lmp(ev)
        np.testing.assert_allclose(ev, 1 + ref["D"], rtol=1e-8)
        h.close()


def test_group_mixed_precision_converges():
    specs = small_uneven(5, seed=7)
    probs = [problem(s_) for s_ in specs]
    hs = [P.Handle.from_spec(s_, taps, precision=P.EDA_MIXED) for s_, (taps, _, _) in zip(specs, probs)]
    with P.Group(hs) as g:
        g.eda_group_set_trajectories([xb for _, xb, _ in probs], [y for _, _, y in probs])
        g.eda_group_sketch()
        g.eda_group_build_lmp()
        g.eda_group_autotune()
        T = g.total_members
        dz = [np.zeros((s_.n_members, s_.n)) for s_ in specs]
        it = np.zeros(T, np.int32)
        rr = np.zeros(T)
        st = np.zeros(T, np.int32)
        g.eda_group_solve(1e-6, 5000, True, dz, it, rr, st)
    for h in hs:
        h.close()
    assert (st == P.EDA_CONVERGED).all()
    # FP64 true residuals at the tolerance; error bounded by the residual
    assert (rr <= 1e-6).all()
    for s_, (taps, xb, y), z in zip(specs, probs, dz):
        traj = O.member_trajectories(s_, xb)
        b = O.rhs(s_, traj, O.innovations(s_, traj, y), taps)
        ref = O.pcg(lambda V: O.hvp(s_, traj, V, taps), b, tol=1e-13, maxit=5000)["x"]
        e = np.linalg.norm(z - ref, axis=1)
        assert (e <= 1.01e-6 * np.linalg.norm(b, axis=1) + 1e-12).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_maxit_is_a_budget_per_member(precision):
    # an easy problem (short window) and a hard one (long window, larger
    # Hessian eigenvalues) in one group: with a budget the hard problem
    # cannot meet, the easy problem's members must still converge, and every
    # member's count stays within the budget
    easy = S.spec_small(64, 6, 4, every_var=2, every_step=2, length_scale=2.0, seed=1)
    hard = S.spec_small(200, 60, 4, every_var=1, every_step=1, length_scale=6.0, seed=2)
    specs = [easy, hard]
    for s_ in specs:
        s_.spinup = 300
    probs = [problem(s_) for s_ in specs]
    prec = P.EDA_FP64 if precision == "fp64" else P.EDA_MIXED
    hs = [P.Handle.from_spec(s_, taps, precision=prec) for s_, (taps, _, _) in zip(specs, probs)]
    # each problem alone: the budget lies between what they need
    need = []
    for s_, (taps, xb, y) in zip(specs, probs):
        with P.Handle.from_spec(s_, taps, precision=prec) as h:
            h.eda_set_trajectory(xb, y)
            itk = np.zeros(s_.n_members, np.int32)
            h.eda_solve_batch(1e-8, 20000, None, False, np.zeros((s_.n_members, s_.n)), itk)
            need.append(int(itk.max()))
    assert need[1] > need[0] + 10, need
    budget = (need[0] + need[1]) // 2
    with P.Group(hs) as g:
        g.eda_group_set_trajectories([xb for _, xb, _ in probs], [y for _, _, y in probs])
        T = g.total_members
        it = np.zeros(T, np.int32)
        rr = np.zeros(T)
        st = np.zeros(T, np.int32)
        g.eda_group_solve(1e-8, budget, False, None, it, rr, st)
    for h in hs:
        h.close()
    m0 = easy.n_members
    assert (st[m0:] == P.EDA_MAXIT).any(), "the hard problem should not converge within the budget"
    assert (st[:m0] == P.EDA_CONVERGED).all() and (rr[:m0] <= 1e-8).all(), (st, rr, it, budget)
    assert (it <= budget).all()
