"""Checkpointed trajectory (ckpt_every = c > 0): the store keeps x_0, x_c,
x_2c, ... of every member, and the Hessian-product and right-hand-side
sweeps recompute each c-step segment from its checkpoint on the chip
(multi-launch tiles with the wider halo that recomputation needs).  The
products, right-hand sides and solutions must match the oracle (which
stores nothing: it recomputes nothing) as the full store does."""
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


def oracle_setup(spec, taps, xb, y):
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    return traj, b


# window not a multiple of c (a short last segment), observations at t = 0
# and at the window end, ragged n, n spanning several tiles
CASES = [
    (S.spec_small(997, 13, 4, every_var=3, every_step=3, length_scale=3.0, seed=31), 4),
    (S.spec_small(3000, 24, 5, every_var=2, every_step=2, length_scale=6.0, seed=32), 8),
    (S.spec_small(600, 9, 3, every_var=1, every_step=1, length_scale=2.0, seed=33), 1),
    (S.spec_small(4096, 20, 3, every_var=2, every_step=4, length_scale=8.0, seed=34), 6),
]


@pytest.mark.parametrize("spec,c", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_checkpointed_hvp_and_rhs_match_the_oracle(spec, c):
    spec = replace(spec, ckpt_every=c, spinup=50)
    taps, xb, y = problem(spec)
    traj, b = oracle_setup(spec, taps, xb, y)
    rng = np.random.default_rng(c)
    ncol = 2 * spec.n_members + 1
    cols = rng.integers(0, spec.n_members, ncol).astype(np.int32)
    V = rng.standard_normal((ncol, spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        plan = h.eda_sweep_plan(fp64=True)
        assert plan["kind"] == "multi-launch" and plan["K"] == c and plan["halo"] == 19 * c + 8
        rhs = np.zeros_like(b)
        h.eda_set_trajectory(xb, y, rhs)
        assert rowrel(rhs, b).max() < 1e-11
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-11
        h.eda_autotune(0)  # only checkpointed plans of K = c are candidates
        assert h.eda_sweep_plan(fp64=True)["K"] == c
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-11
    with P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-4


def test_checkpointed_solve_matches_the_full_store():
    # the same batched solve with and without checkpoints: equal up to the
    # rounding of the recomputed states, at equal iteration counts
    spec = S.spec_tiny(seed=16)
    taps, xb, y = problem(spec)
    ref = O.eda_pipeline(spec, xb, y, taps, tol=0, maxit=1, fixed_iters=1)
    out = {}
    for c in (0, 5):
        with P.Handle.from_spec(replace(spec, ckpt_every=c), taps, precision=P.EDA_FP64) as h:
            h.eda_set_trajectory(xb, y)
            h.eda_set_lmp(np.ascontiguousarray(ref["S"].T), 1 + ref["D"])
            dz = np.zeros((spec.n_members, spec.n))
            h.eda_solve_batch(0.0, 8, None, True, dz)
            out[c] = dz
    assert rowrel(out[5], out[0]).max() < 1e-10


def test_checkpointed_handles_are_not_grouped_and_bad_periods_refused():
    spec = replace(S.spec_tiny(seed=17), ckpt_every=4)
    taps, xb, y = problem(spec)
    with P.Handle.from_spec(spec, taps) as h:
        with pytest.raises(P.EdaError):
            P.Group([h])
    with pytest.raises(P.EdaError):
        P.Handle.from_spec(replace(spec, ckpt_every=-1), taps)


def test_full_size_scale_checkpointed_every_8_steps():
    # the n = 65536, 96-step, 81-member workload with a checkpoint every 8
    # steps (13 stored states per member instead of 97): sampled products
    # and right-hand sides against the oracle
    spec = replace(S.spec_scale(seed=0), ckpt_every=8, spinup=100)
    taps, xb, y = problem(spec)
    sample = np.array([0, 37, 80], dtype=np.int32)
    traj = O.member_trajectories(spec, xb[sample])
    b = O.rhs(spec, traj, O.innovations(spec, traj, y[sample]), taps)
    V = np.random.default_rng(22).standard_normal((len(sample), spec.n))
    ref = O.hvp(spec, traj, V, taps)
    # three PCG iterations (no LMP) of the sampled members against the oracle
    K = 3
    oref = O.pcg(lambda W: O.hvp(spec, traj, W, taps), b, tol=0, maxit=K, fixed_iters=K)["x"]
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        rhs = np.zeros((spec.n_members, spec.n))
        h.eda_set_trajectory(xb, y, rhs)
        assert rowrel(rhs[sample], b).max() < 1e-10
        HV = np.zeros_like(V)
        h.eda_hvp(sample, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-10
        dz = np.zeros((spec.n_members, spec.n))
        h.eda_solve_batch(0.0, K, None, False, dz)
        assert rowrel(dz[sample], oref).max() < 1e-10
    with P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        HV = np.zeros_like(V)
        h.eda_hvp(sample, V, HV, True)
        e32 = rowrel(HV, ref).max()
        print("checkpointed FP32 sweep HVP rel err at n=65536, N=96: %.3e" % e32)
        assert e32 < 1e-3
