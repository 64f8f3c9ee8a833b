"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Inputs come from the seeded draws and the oracle's identical twin; expected
values from the oracle.  FP64 path: 1e-10 relative (Hessian products,
right-hand sides, solutions at equal iteration counts); mixed path: the error
against the oracle is reported and bounded.
"""
from dataclasses import replace

import numpy as np
import pytest

import eda_synth as S
import oracle as O
from helpers import env, problem, rel, rowrel

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_23571_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make(spec, taps, precision=P.EDA_FP64, **kw):
    return P.Handle.from_spec(spec, taps, precision=precision, **kw)


def oracle_setup(spec, taps, xb, y):
    traj = O.member_trajectories(spec, xb)
    d = O.innovations(spec, traj, y)
    b = O.rhs(spec, traj, d, taps)
    return traj, d, b


SMALL = [
    S.spec_small(40, 20, 11, every_step=4, length_scale=2.0),   # the n=40 tiny workload
    S.spec_small(97, 13, 5, every_var=3, every_step=3, length_scale=3.0, seed=1),  # ragged
    S.spec_small(5, 6, 3, every_var=1, every_step=1, length_scale=0.7, seed=2),    # minimal n
    S.spec_small(300, 16, 7, every_var=2, every_step=2, length_scale=8.0, seed=3),
]


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
def test_twin_matches_oracle_without_spinup(spec):
    spec = replace(spec, spinup=3)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    dr = S.draws(spec)
    _, xb_o, y_o = O.twin(spec, dr, taps)
    x_spin0 = spec.F + spec.spin_sigma * dr.eta_spin
    with make(spec, taps) as h:
        xb = np.zeros((spec.n_members, spec.n))
        y = np.zeros((spec.n_members, spec.p))
        h.eda_twin(np.ascontiguousarray(x_spin0), spec.spinup, dr.eta_b, dr.eta_o, xb, y)
    assert rel(xb, xb_o) < 1e-13
    assert rel(y, y_o) < 1e-13


@pytest.mark.parametrize("store", [1, 0], ids=["stored-stages", "recomputed-stages"])
@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
def test_rhs_and_hvp_fp64(spec, store):
    # the FP64 sweeps read the RK4 stage states stored with the trajectory,
    # or recompute them (EDA_STAGE_STORE=0); FP32 sweeps always recompute
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    rng = np.random.default_rng(7)
    ncol = 2 * spec.n_members + 1
    cols = rng.integers(0, spec.n_members, ncol).astype(np.int32)
    V = rng.standard_normal((ncol, spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    refA = O.hvp(spec, traj[cols], V, taps, identity=False)
    with env(EDA_STAGE_STORE=store):
        with make(spec, taps) as h:
            rhs = np.zeros_like(b)
            h.eda_set_trajectory(xb, y, rhs)
            assert rowrel(rhs, b).max() < 1e-11
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-11
            h.eda_hvp(cols, V, HV, False)
            assert rowrel(HV, refA).max() < 1e-10
        with make(spec, taps, precision=P.EDA_MIXED) as h:
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-4


@pytest.mark.parametrize("cs", [2, 3, 5])
def test_hvp_fp64_cluster_split(cs):
    # the same column split over a cluster of CTAs exchanging halos
    spec = S.spec_small(600, 24, 4, every_var=2, every_step=3, length_scale=4.0, seed=5)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    rng = np.random.default_rng(cs)
    cols = np.array([0, 1, 2, 3, 0], dtype=np.int32)
    V = rng.standard_normal((len(cols), spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    for K in (1, 3, 8):
        with env(EDA_SWEEP_CS64=cs, EDA_SWEEP_K=K):
            with make(spec, taps) as h:
                rhs = np.zeros_like(b)
                h.eda_set_trajectory(xb, y, rhs)
                assert rowrel(rhs, b).max() < 1e-11, (cs, K)
                HV = np.zeros_like(V)
                h.eda_hvp(cols, V, HV, True)
                assert rowrel(HV, ref).max() < 1e-11, (cs, K)


@pytest.mark.parametrize("c64,c32", [(2, 4), (4, 8), (4, 2)])
def test_hvp_with_each_run_length(c64, c32):
    # every instantiated run length (values per thread) of the sweep kernel,
    # alone and split over a cluster, FP64 against the oracle and the FP32
    # sweep within single-precision error
    spec = S.spec_small(600, 24, 4, every_var=2, every_step=3, length_scale=4.0, seed=15)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    cols = np.array([0, 1, 2, 3, 2], dtype=np.int32)
    V = np.random.default_rng(4).standard_normal((len(cols), spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    for cs in (1, 3):
        with env(EDA_SWEEP_C64=c64, EDA_SWEEP_C32=c32, EDA_SWEEP_CS64=cs, EDA_SWEEP_CS32=cs):
            with make(spec, taps) as h:
                rhs = np.zeros_like(b)
                h.eda_set_trajectory(xb, y, rhs)
                assert rowrel(rhs, b).max() < 1e-11, (c64, cs)
                HV = np.zeros_like(V)
                h.eda_hvp(cols, V, HV, True)
                assert rowrel(HV, ref).max() < 1e-11, (c64, cs)
            with make(spec, taps, precision=P.EDA_MIXED) as h:
                h.eda_set_trajectory(xb, y)
                HV = np.zeros_like(V)
                h.eda_hvp(cols, V, HV, True)
                assert rowrel(HV, ref).max() < 1e-4, (c32, cs)


def _ml_spec(n, seed):
    # observations at t = 0 and t = N as well as inside the window
    N = 13
    steps = np.array([0, 3, 6, 9, 12, 13], dtype=np.int32)
    idx1 = np.arange(0, n, 2, dtype=np.int32)
    return S.Spec(n=n, nsteps=N, obs_steps=steps,
                  obs_ptr=(np.arange(len(steps) + 1) * len(idx1)).astype(np.int32),
                  obs_idx=np.tile(idx1, len(steps)), sigma_o=1.0, sigma_b=1.0,
                  length_scale=4.0, n_members=5, ell=4, k=4, spinup=5, seed=seed,
                  name="l96_n%d_w13_m5" % n)


# (n, threads per CTA, launch length K): FP64 tiles of 256 - 2(8K + 8) and
# FP32 tiles of 512 - 2(8K + 8) owned points, so that one column spans 2 to 6
# tiles with a ragged last tile; n = 997 also disables the 16-byte loads
ML_CASES = [(600, 64, 2), (997, 64, 3), (1000, 128, 1)]


@pytest.mark.parametrize("n,threads,K", ML_CASES)
def test_multi_launch_sweeps_match_oracle(n, threads, K):
    # sweeps of states too large for one cluster run as chains of K-step
    # launches whose state passes through global memory; forced here at
    # small n: twin (spin-up and trajectories), right-hand sides, products
    # with and without the identity, the sketch and the LMP
    spec = _ml_spec(n, seed=n)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    dr = S.draws(spec)
    _, xb, y = O.twin(spec, dr, taps)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    rng = np.random.default_rng(n)
    cols = np.array([0, 3, 1, 4, 2, 0, 3], dtype=np.int32)
    V = rng.standard_normal((len(cols), spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    refA = O.hvp(spec, traj[cols], V, taps, identity=False)
    with env(EDA_SWEEP_ML=threads, EDA_SWEEP_K=K):
        with make(spec, taps) as h:
            xb_g = np.zeros((spec.n_members, spec.n))
            y_g = np.zeros((spec.n_members, spec.p))
            h.eda_twin(np.ascontiguousarray(spec.F + spec.spin_sigma * dr.eta_spin), spec.spinup,
                       dr.eta_b, dr.eta_o, xb_g, y_g)
            assert rel(xb_g, xb) < 1e-13 and rel(y_g, y) < 1e-13
            rhs = np.zeros_like(b)
            h.eda_set_trajectory(xb, y, rhs)
            assert rowrel(rhs, b).max() < 1e-11
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-11
            h.eda_hvp(cols, V, HV, False)
            assert rowrel(HV, refA).max() < 1e-10
            h.eda_sketch()
            ev = np.zeros(spec.k)
            h.eda_build_lmp(ev)
            ro = O.eda_pipeline(spec, xb, y, taps, tol=1e-6, maxit=200)
            np.testing.assert_allclose(ev, 1 + ro["D"], rtol=1e-9)
        with make(spec, taps, precision=P.EDA_MIXED) as h:
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-4
            h.eda_sketch()
            h.eda_build_lmp()
            dz = np.zeros_like(b)
            rr = np.zeros(spec.n_members)
            st = np.zeros(spec.n_members, np.int32)
            h.eda_solve_batch(1e-8, 500, None, True, dz, None, rr, st)
            assert (st == P.EDA_CONVERGED).all() and (rr <= 1e-8).all()
            exact = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=500)["x"]
            bn = np.linalg.norm(b, axis=1)
            assert (np.linalg.norm(dz - exact, axis=1) <= rr * bn * (1 + 1e-6) + 1e-12).all()


def _subset_spec(n, seed):
    # a random subset of the variables observed (the same at every step), with
    # observations at t = 0 and N as well
    rng = np.random.default_rng(seed)
    idx1 = np.sort(rng.choice(n, size=int(0.3 * n), replace=False)).astype(np.int32)
    steps = np.array([0, 2, 4, 7, 9, 12, 13], dtype=np.int32)
    return S.Spec(n=n, nsteps=13, obs_steps=steps,
                  obs_ptr=(np.arange(len(steps) + 1) * len(idx1)).astype(np.int32),
                  obs_idx=np.tile(idx1, len(steps)), sigma_o=0.7, sigma_b=1.0,
                  length_scale=5.0, n_members=5, ell=4, k=4, spinup=5, seed=seed,
                  name="l96_n%d_w13_m5_subset" % n)


def _varied_spec(n, seed):
    # a different observation set at every observation step (all variables,
    # every third, random subsets, every second), including t = 0 and t = N
    rng = np.random.default_rng(seed)
    steps = np.array([0, 1, 4, 7, 12, 13], dtype=np.int32)
    sets = [np.arange(n), np.arange(0, n, 3), np.sort(rng.choice(n, int(0.3 * n), replace=False)),
            np.arange(n), np.sort(rng.choice(n, int(0.5 * n), replace=False)), np.arange(1, n, 2)]
    ptr = np.concatenate([[0], np.cumsum([len(x) for x in sets])]).astype(np.int32)
    return S.Spec(n=n, nsteps=13, obs_steps=steps, obs_ptr=ptr,
                  obs_idx=np.concatenate(sets).astype(np.int32), sigma_o=0.8, sigma_b=1.0,
                  length_scale=4.0, n_members=4, ell=3, k=3, spinup=5, seed=seed,
                  name="l96_n%d_w13_m4_varied" % n)


# (n, cluster size, refresh period, values per thread FP64, FP32): odd n puts
# the wrap n-1 -> 0 of the last CTA's region inside a thread's run
VARIED_OBS_CASES = [(997, 2, 4, 4, 8), (997, 3, 1, 2, 4), (1001, 3, 4, 4, 4), (1001, 2, 2, 2, 8), (998, 3, 2, 4, 2)]


@pytest.mark.parametrize("n,cs,K,c64,c32", VARIED_OBS_CASES)
def test_cluster_plans_with_varied_observation_sets(n, cs, K, c64, c32):
    # cluster plans over an observation network that changes from step to
    # step (dense, sparse, random subsets, t = 0 and t = N) with a ragged n:
    # the right-hand side and the products with and without the identity
    # against the oracle, stage states stored or recomputed, and FP32
    spec = _varied_spec(n, seed=n + cs)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    cols = np.array([0, 3, 1, 2, 0], dtype=np.int32)
    V = np.random.default_rng(n * cs).standard_normal((len(cols), spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    refA = O.hvp(spec, traj[cols], V, taps, identity=False)
    with env(EDA_SWEEP_CS64=cs, EDA_SWEEP_CS32=cs, EDA_SWEEP_K=K, EDA_SWEEP_C64=c64, EDA_SWEEP_C32=c32):
        for store in (1, 0):
            with env(EDA_STAGE_STORE=store):
                with make(spec, taps) as h:
                    assert h.eda_sweep_plan(True)["kind"] == "cluster"
                    rhs = np.zeros_like(b)
                    h.eda_set_trajectory(xb, y, rhs)
                    assert rowrel(rhs, b).max() < 1e-11, store
                    HV = np.zeros_like(V)
                    h.eda_hvp(cols, V, HV, True)
                    assert rowrel(HV, ref).max() < 1e-11, store
                    h.eda_hvp(cols, V, HV, False)
                    assert rowrel(HV, refA).max() < 1e-10, store
        with make(spec, taps, precision=P.EDA_MIXED) as h:
            assert h.eda_sweep_plan(False)["kind"] == "cluster"
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-4
            h.eda_hvp(cols, V, HV, False)
            assert rowrel(HV, refA).max() < 1e-4


# (n, cluster size, refresh period, values per lane FP64, FP32, observation network)
WARP_CASES = [(1000, 2, 8, 4, 8, "regular"), (1000, 3, 4, 2, 4, "regular"),
              (997, 3, 8, 4, 4, "subset"), (2048, 5, 4, 2, 8, "subset")]


@pytest.mark.parametrize("n,cs,K,c64,c32,net", WARP_CASES)
def test_warp_tiled_sweeps_match_oracle(n, cs, K, c64, c32, net):
    # the warp-tiled Hessian-product kernel (shuffle stencils, warp halos
    # refreshed every step, cluster halos every K steps): products with and
    # without the identity, the sketch and LMP, and a preconditioned solve
    # whose p.q comes from the sweep epilogue
    spec = _ml_spec(n, seed=n) if net == "regular" else _subset_spec(n, seed=n)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    cols = np.array([0, 3, 1, 4, 2, 0, 3], dtype=np.int32)
    V = np.random.default_rng(n + cs).standard_normal((len(cols), spec.n))
    ref = O.hvp(spec, traj[cols], V, taps)
    refA = O.hvp(spec, traj[cols], V, taps, identity=False)
    with env(EDA_SWEEP_WARP=1, EDA_SWEEP_CS64=cs, EDA_SWEEP_CS32=cs, EDA_SWEEP_K=K,
             EDA_SWEEP_C64=c64, EDA_SWEEP_C32=c32):
        with make(spec, taps) as h:
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-11
            h.eda_hvp(cols, V, HV, False)
            assert rowrel(HV, refA).max() < 1e-10
            h.eda_sketch()
            ev = np.zeros(spec.k)
            h.eda_build_lmp(ev)
            ro = O.eda_pipeline(spec, xb, y, taps, tol=1e-6, maxit=200)
            np.testing.assert_allclose(ev, 1 + ro["D"], rtol=1e-9)
            dz = np.zeros_like(b)
            rr = np.zeros(spec.n_members)
            st = np.zeros(spec.n_members, np.int32)
            h.eda_solve_batch(1e-10, 500, None, True, dz, None, rr, st)
            assert (st == P.EDA_CONVERGED).all()
            exact = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=500)["x"]
            bn = np.linalg.norm(b, axis=1)
            assert (np.linalg.norm(dz - exact, axis=1) <= 1.5e-10 * bn).all()
        with make(spec, taps, precision=P.EDA_MIXED) as h:
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-4
            h.eda_sketch()
            h.eda_build_lmp()
            dz = np.zeros_like(b)
            rr = np.zeros(spec.n_members)
            st = np.zeros(spec.n_members, np.int32)
            h.eda_solve_batch(1e-8, 500, None, True, dz, None, rr, st)
            assert (st == P.EDA_CONVERGED).all() and (rr <= 1e-8).all()


def test_warp_tiled_full_size_batched_hvp():
    # the n=4096, 64-step, 51-member workload on the warp-tiled kernel
    spec = replace(S.spec_batched(seed=0), spinup=200)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    cols = np.arange(spec.n_members, dtype=np.int32)
    V = np.random.default_rng(12).standard_normal((spec.n_members, spec.n))
    ref = O.hvp(spec, traj, V, taps)
    with env(EDA_SWEEP_WARP=1, EDA_SWEEP_CS64=5, EDA_SWEEP_CS32=5):
        with make(spec, taps) as h:
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-10
        with make(spec, taps, precision=P.EDA_MIXED) as h:
            h.eda_set_trajectory(xb, y)
            HV = np.zeros_like(V)
            h.eda_hvp(cols, V, HV, True)
            assert rowrel(HV, ref).max() < 1e-4


def test_autotuned_tiling_keeps_parity():
    # the autotuner times cluster and multi-launch tilings and keeps the
    # fastest; whichever it keeps must give the same products
    spec = S.spec_small(2500, 16, 6, every_var=2, every_step=2, length_scale=6.0, seed=9)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    cols = np.arange(spec.n_members, dtype=np.int32)
    V = np.random.default_rng(2).standard_normal((spec.n_members, spec.n))
    ref = O.hvp(spec, traj, V, taps)
    with make(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        assert h.eda_autotune(3) > 0
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-4
        for fp64, runs in ((False, (4, 8)), (True, (2, 4))):
            plan = h.eda_sweep_plan(fp64)
            assert plan["kind"] in ("cluster", "multi-launch", "warp") and plan["C"] in runs
            assert plan["K"] >= 1 and plan["threads"] % 32 == 0 and plan["ctas_per_vector"] >= 1
            if plan["kind"] != "warp":
                # CTAs x owned points cover the state; each tile carries its
                # halo of 8K + 8 points (the K-step reach) at both ends
                assert plan["halo"] == 8 * plan["K"] + 8
                assert plan["ctas_per_vector"] * plan["owned"] >= spec.n
                assert plan["owned"] + 2 * plan["halo"] <= plan["threads"] * plan["C"]
    with make(spec, taps) as h:
        h.eda_set_trajectory(xb, y)
        assert h.eda_autotune(1) > 0
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-11
        with pytest.raises(P.EdaError):
            h.eda_sweep_plan(False)  # an FP64 handle has no FP32 sweep


def test_hvp_obs_at_window_ends():
    # observations at t = 0 and t = N exercise the first gather and the first
    # injection of the sweeps
    n, N = 64, 9
    steps = np.array([0, 4, 9], dtype=np.int32)
    idx1 = np.arange(0, n, 3, dtype=np.int32)
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps,
                  obs_ptr=(np.arange(4) * len(idx1)).astype(np.int32),
                  obs_idx=np.tile(idx1, 3), sigma_o=0.5, sigma_b=1.0, length_scale=2.5,
                  n_members=3, ell=2, k=2)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    V = np.random.default_rng(1).standard_normal((3, n))
    cols = np.arange(3, dtype=np.int32)
    with make(spec, taps) as h:
        rhs = np.zeros_like(b)
        h.eda_set_trajectory(xb, y, rhs)
        assert rowrel(rhs, b).max() < 1e-11
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, O.hvp(spec, traj, V, taps)).max() < 1e-11


def oracle_self_sensitivity(spec, traj, b, taps, S_, c_, K, seed=0):
    """How far the oracle's own K-iteration PCG iterate moves when b is
    perturbed by 1e-16 relative: CG amplifies rounding on some members, and
    two correct FP64 implementations cannot agree below this level."""
    P_ = lambda R: O.lmp_apply(S_, c_, R)
    a = O.pcg(lambda V: O.hvp(spec, traj, V, taps), b, P_, tol=0, maxit=K, fixed_iters=K)
    bp = b * (1 + 1e-16 * np.random.default_rng(seed).standard_normal(b.shape))
    c = O.pcg(lambda V: O.hvp(spec, traj, V, taps), bp, P_, tol=0, maxit=K, fixed_iters=K)
    return rowrel(c["x"], a["x"])


def test_sketch_lmp_and_solve_fp64_tiny():
    spec = S.spec_tiny(seed=4)
    taps, xb, y = problem(spec)
    # equal iteration counts no larger than the fewest any member needs to
    # reach 1e-6, so that no member is iterating on rounding noise
    Kmin = int(O.eda_pipeline(spec, xb, y, taps, tol=1e-6, maxit=100)["iters"].min())
    with make(spec, taps) as h:
        ref = O.eda_pipeline(spec, xb, y, taps, tol=0, maxit=Kmin, fixed_iters=Kmin)
        rhs = np.zeros_like(ref["b"])
        h.eda_set_trajectory(xb, y, rhs)
        Yg = np.zeros((spec.ell, spec.n))
        h.eda_sketch(None, 1, Yg)
        assert rel(Yg, ref["Y"].T) < 1e-11
        ev = np.zeros(spec.k)
        Sg = np.zeros((spec.k, spec.n))
        h.eda_build_lmp(ev, Sg)
        np.testing.assert_allclose(ev, 1 + ref["D"], rtol=1e-9)
        # LMP action (sign/rotation invariant): S diag(c) S^T
        Pg = (Sg.T * ref["c"]) @ Sg
        Po = (ref["S"] * ref["c"]) @ ref["S"].T
        assert np.linalg.norm(Pg - Po) <= 1e-8 * np.linalg.norm(Po)
        # PCG parity with one preconditioner on both sides: the Nystrom
        # factors agree only to ~eps * cond(Phi^T A Phi) ~ 1e-8, and CG
        # amplifies preconditioner differences, so the oracle's LMP is loaded
        h.eda_set_lmp(np.ascontiguousarray(ref["S"].T), 1 + ref["D"])
        for K in (8, Kmin):
            refK = O.pcg(lambda V: O.hvp(spec, ref["traj"], V, taps), ref["b"],
                         lambda R: O.lmp_apply(ref["S"], ref["c"], R), tol=0, maxit=K, fixed_iters=K)
            sens = oracle_self_sensitivity(spec, ref["traj"], ref["b"], taps, ref["S"], ref["c"], K)
            dz = np.zeros_like(ref["b"])
            it = np.zeros(spec.n_members, np.int32)
            rr = np.zeros(spec.n_members)
            st = np.zeros(spec.n_members, np.int32)
            h.eda_solve_batch(0.0, K, None, True, dz, it, rr, st)
            assert (it == K).all()
            err = rowrel(dz, refK["x"])
            # the 1e-10 bar on every member whose oracle iterate moves by less
            # than 1e-12 under a 1e-16 perturbation of b (elsewhere CG
            # amplifies rounding beyond what two FP64 codes can agree on)
            calm = sens < 1e-12
            assert calm.sum() >= spec.n_members // 2, (K, sens)
            assert (err[calm] < 1e-10).all(), (K, err, sens)
            np.testing.assert_allclose(rr[calm], refK["relres"][calm], rtol=1e-6)
        # converged: both solved to relative residual 1e-13, 1e-10 on every member
        exact = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=300)["x"]
        dz = np.zeros_like(ref["b"])
        h.eda_solve_batch(1e-13, 300, None, True, dz)
        assert rowrel(dz, exact).max() < 1e-10


def test_solve_tolerance_stopped_fp64_tiny():
    spec = S.spec_tiny(seed=5)
    taps, xb, y = problem(spec)
    ref = O.eda_pipeline(spec, xb, y, taps, tol=1e-6, maxit=100)
    exact = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=300)["x"]
    with make(spec, taps) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_set_lmp(np.ascontiguousarray(ref["S"].T), 1 + ref["D"])
        dz = np.zeros_like(ref["b"])
        it = np.zeros(spec.n_members, np.int32)
        rr = np.zeros(spec.n_members)
        st = np.zeros(spec.n_members, np.int32)
        h.eda_solve_batch(1e-6, 100, None, True, dz, it, rr, st)
        assert (st == P.EDA_CONVERGED).all()
        assert (rr <= 1e-6).all()
        # stopping counts: +-1 of the oracle's, widened on members whose own
        # count moves when b is perturbed by 1e-16 (CG rounding sensitivity)
        lo, hi = ref["iters"].copy(), ref["iters"].copy()
        traj = ref["traj"]
        for sd in range(10):
            bp = ref["b"] * (1 + 1e-16 * np.random.default_rng(sd).standard_normal(ref["b"].shape))
            c2 = O.pcg(lambda V: O.hvp(spec, traj, V, taps), bp,
                       lambda R: O.lmp_apply(ref["S"], ref["c"], R), tol=1e-6, maxit=100)["iters"]
            lo, hi = np.minimum(lo, c2), np.maximum(hi, c2)
        assert ((it >= lo - 1) & (it <= hi + 1)).all(), (it, lo, hi)
        # and with the LMP the library builds itself: converged, error bound
        h.eda_sketch()
        h.eda_build_lmp()
        h.eda_solve_batch(1e-6, 100, None, True, dz, it, rr, st)
    assert (st == P.EDA_CONVERGED).all()
    assert np.abs(it - ref["iters"]).max() <= 3
    assert (rr <= 1e-6).all()
    # ||dz - dz*|| <= ||r|| since lambda_min(I + A) >= 1
    err = np.linalg.norm(dz - exact, axis=1)
    assert (err <= rr * np.linalg.norm(ref["b"], axis=1) * (1 + 1e-6) + 1e-12).all()


def test_solve_without_lmp_and_with_x0():
    spec = S.spec_small(97, 13, 5, every_var=3, every_step=3, length_scale=3.0, seed=6)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    x0 = np.random.default_rng(3).standard_normal(b.shape) * 0.1
    ref = O.pcg(lambda V: O.hvp(spec, traj, V, taps), b, tol=0, maxit=9, x0=x0, fixed_iters=9)
    with make(spec, taps) as h:
        h.eda_set_trajectory(xb, y)
        dz = np.zeros_like(b)
        h.eda_solve_batch(0.0, 9, x0, False, dz)
    assert rowrel(dz, ref["x"]).max() < 1e-10


def test_mixed_precision_tiny_reports_error():
    spec = S.spec_tiny(seed=6)
    taps, xb, y = problem(spec)
    exact = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=300)
    with make(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_sketch()
        h.eda_build_lmp()
        dz = np.zeros_like(exact["b"])
        it = np.zeros(spec.n_members, np.int32)
        rr = np.zeros(spec.n_members)
        st = np.zeros(spec.n_members, np.int32)
        h.eda_solve_batch(1e-6, 200, None, True, dz, it, rr, st)
    err = rowrel(dz, exact["x"])
    print("mixed tiny: max rel err %.3e, iters %s, true relres max %.3e" % (err.max(), it, rr.max()))
    assert (st == P.EDA_CONVERGED).all()
    assert (rr <= 1e-6).all()
    # the FP64 true residual bounds the error: ||e|| <= ||r|| (lambda_min >= 1)
    bn = np.linalg.norm(exact["b"], axis=1)
    assert (np.linalg.norm(dz - exact["x"], axis=1) <= rr * bn * (1 + 1e-6) + 1e-12).all()


def test_hvp_device_tensors_and_empty_batch():
    import torch
    spec = S.spec_small(40, 20, 3, every_step=4)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    dev = torch.device("cuda:0")
    with make(spec, taps) as h:
        h.eda_set_trajectory(torch.tensor(xb, device=dev), torch.tensor(y, device=dev))
        V = torch.randn(4, spec.n, dtype=torch.float64, device=dev)
        HV = torch.empty_like(V)
        cols = torch.tensor([2, 0, 1, 2], dtype=torch.int32, device=dev)
        h.eda_hvp(cols, V, HV, True)
        torch.cuda.synchronize()
        ref = O.hvp(spec, traj[[2, 0, 1, 2]], V.cpu().numpy(), taps)
        assert rowrel(HV.cpu().numpy(), ref).max() < 1e-11
        h.eda_hvp(np.zeros(0, np.int32), np.zeros((0, spec.n)), np.zeros((0, spec.n)), True)


def test_errors_are_reported():
    spec = S.spec_small(40, 20, 3, every_step=4)
    taps, xb, y = problem(spec)
    with make(spec, taps) as h:
        with pytest.raises(P.EdaError) as e:
            h.eda_sketch()
        assert e.value.code == P.EDA_ERR_STATE
        bad = xb.copy()
        bad[1, 3] = np.nan
        with pytest.raises(P.EdaError) as e:
            h.eda_set_trajectory(bad, y)
        assert e.value.code == P.EDA_ERR_NUMERIC
    with pytest.raises(P.EdaError) as e:
        P.Handle.from_spec(spec, taps, n=3)
    assert e.value.code == P.EDA_ERR_INVALID


def test_full_size_batched_hvp_and_rhs_fp64():
    # the n=4096, 64-step, 51-member workload: RHS of every member and one
    # batched product (members' own trajectories) against the oracle
    spec = replace(S.spec_batched(seed=0), spinup=200)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    rng = np.random.default_rng(11)
    cols = np.arange(spec.n_members, dtype=np.int32)
    V = rng.standard_normal((spec.n_members, spec.n))
    ref = O.hvp(spec, traj, V, taps)
    with make(spec, taps) as h:
        rhs = np.zeros_like(b)
        h.eda_set_trajectory(xb, y, rhs)
        assert rowrel(rhs, b).max() < 1e-10
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-10
    with make(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        HV = np.zeros_like(V)
        h.eda_hvp(cols, V, HV, True)
        e32 = rowrel(HV, ref).max()
        print("FP32 sweep HVP rel err at n=4096, N=64: %.3e" % e32)
        assert e32 < 1e-4


@pytest.mark.slow
def test_full_size_scale_hvp_sampled_columns():
    # the n=65536, 96-step, 81-member workload (multi-launch tiling): products
    # of a sample of members on their own trajectories against the oracle,
    # column by column, and the right-hand sides of the same members
    spec = replace(S.spec_scale(seed=0), ckpt_every=0, spinup=100)
    taps, xb, y = problem(spec)
    sample = np.array([0, 37, 80], dtype=np.int32)
    traj = O.member_trajectories(spec, xb[sample])
    d = O.innovations(spec, traj, y[sample])
    b = O.rhs(spec, traj, d, taps)
    V = np.random.default_rng(21).standard_normal((len(sample), spec.n))
    ref = O.hvp(spec, traj, V, taps)
    with make(spec, taps) as h:
        rhs = np.zeros((spec.n_members, spec.n))
        h.eda_set_trajectory(xb, y, rhs)
        assert rowrel(rhs[sample], b).max() < 1e-10
        HV = np.zeros_like(V)
        h.eda_hvp(sample, V, HV, True)
        assert rowrel(HV, ref).max() < 1e-10
    with make(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        HV = np.zeros_like(V)
        h.eda_hvp(sample, V, HV, True)
        e32 = rowrel(HV, ref).max()
        print("FP32 sweep HVP rel err at n=65536, N=96: %.3e" % e32)
        assert e32 < 1e-3


def test_rank_deficient_sketch_uses_the_truncated_eigendecomposition():
    # a length scale comparable to n leaves B, and so Gamma, numerically rank
    # deficient: Cholesky and the shift both break down and Algorithm 1 is
    # completed with truncated eigendecompositions (Appendix B).  The
    # approximation A_N = Y W^+ Y^T must match the oracle's on its
    # significant part, and the preconditioned solve still converges.
    n, N = 41, 10
    steps, ptr, idx = S.regular_obs(n, N, 3, 2)
    spec = S.Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=idx, sigma_o=1.0,
                  sigma_b=1.0, length_scale=7.6, n_members=33, ell=32, k=31, spinup=300)
    taps, xb, y = problem(spec)
    ref = O.eda_pipeline(spec, xb, y, taps, tol=1e-6, maxit=500)
    with make(spec, taps) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_sketch()
        ev = np.zeros(spec.k)
        Sg = np.zeros((spec.k, spec.n))
        h.eda_build_lmp(ev, Sg)
        path, rank, shift = h.eda_lmp_info()
        assert path == 2 and shift == 0.0
        # the approximation's rank is below k: orthonormal eigenvectors up to
        # it, zero columns (lambda = 1) beyond
        r = int((ref["D"] > 0).sum())
        assert rank < spec.k and abs(rank - r) <= 1
        np.testing.assert_allclose(Sg[:rank] @ Sg[:rank].T, np.eye(rank), atol=1e-10)
        assert not Sg[rank:].any() and (ev[rank:] == 1.0).all()
        # a truncated pseudo-inverse amplifies rounding by 1/mu: the oracle's
        # own small modes move under a 1e-16 perturbation of b, and two
        # correct implementations agree only to that level (times a margin)
        traj = ref["traj"]
        f = lambda B_: O.apply_A(spec, np.broadcast_to(traj[0:1], (B_.shape[1],) + traj.shape[1:]),
                                 B_.T.copy(), taps).T
        sens = np.zeros(r)
        for sd in range(4):
            bp = ref["b"] * (1 + 1e-16 * np.random.default_rng(sd).standard_normal(ref["b"].shape))
            Dp = O.nystrom(f, O.gamma(bp)[:, : spec.ell], spec.k)[1]
            sens = np.maximum(sens, np.abs(Dp[:r] - ref["D"][:r]) / ref["D"][:r])
        D = ev - 1
        m = min(r, rank)
        err = np.abs(D[:m] - ref["D"][:m]) / ref["D"][:m]
        assert (err <= np.maximum(1e-9, 10.0 * sens[:m])).all(), (err, sens)
        AN_g = (Sg.T * D) @ Sg
        AN_o = (ref["S"] * ref["D"]) @ ref["S"].T
        assert np.linalg.norm(AN_g - AN_o) <= 1e-6 * np.linalg.norm(AN_o)
        dz = np.zeros((spec.n_members, spec.n))
        st = np.zeros(spec.n_members, np.int32)
        rr = np.zeros(spec.n_members)
        h.eda_solve_batch(1e-6, 500, None, True, dz, None, rr, st)
    assert (st == P.EDA_CONVERGED).all() and (rr <= 1e-6).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_control_only_problem_without_lmp(precision):
    # a single member (no perturbed members, so no sketch and no LMP): the
    # row-chunk PCG kernels run with no projections, the sketch is refused,
    # and the solution matches the oracle's
    spec = S.spec_small(97, 12, 1, every_var=3, every_step=3, length_scale=3.0, ell=0, k=0, seed=13)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    exact = O.pcg(lambda V: O.hvp(spec, traj, V, taps), b, tol=1e-13, maxit=2000)["x"]
    prec = P.EDA_FP64 if precision == "fp64" else P.EDA_MIXED
    with make(spec, taps, precision=prec) as h:
        h.eda_set_trajectory(xb, y)
        with pytest.raises(P.EdaError) as e:
            h.eda_sketch()
        assert e.value.code == P.EDA_ERR_INVALID
        dz = np.zeros_like(b)
        rr = np.zeros(1)
        st = np.zeros(1, np.int32)
        h.eda_solve_batch(1e-9, 2000, None, False, dz, None, rr, st)
    assert st[0] == P.EDA_CONVERGED and rr[0] <= 1e-9
    assert np.linalg.norm(dz - exact) <= rr[0] * np.linalg.norm(b) * (1 + 1e-6) + 1e-12


def test_bhalf_apply_matches_the_circulant():
    # the control-variable transform dx = U_B dz (host and device buffers,
    # empty batch) against the oracle's banded circulant
    import torch
    spec = S.spec_small(300, 8, 5, every_var=2, every_step=2, length_scale=8.0, seed=21)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    V = np.random.default_rng(21).standard_normal((7, spec.n))
    ref = O.bhalf_apply(V, taps)
    with make(spec, taps) as h:
        out = np.zeros_like(V)
        h.eda_bhalf_apply(V, out)
        assert rel(out, ref) < 1e-14
        Vd = torch.tensor(V, device="cuda")
        Od = torch.zeros_like(Vd)
        h.eda_bhalf_apply(Vd, Od)
        assert rel(Od.cpu().numpy(), ref) < 1e-14
        h.eda_bhalf_apply(V[:0], out[:0])


def _ctrl_apply(spec, traj, taps):
    ctrl = traj[0:1]

    def apply_ctrl(block):
        tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
        return O.apply_A(spec, tr, block.T.copy(), taps).T
    return apply_ctrl


@pytest.mark.parametrize("q", [1, 2])
@pytest.mark.parametrize("kind", ["psi", "ub_psi", "b_psi"])
def test_sketch_of_a_given_matrix_with_power_passes(kind, q):
    # Algorithm 1 on a caller's sketch matrix: a Gaussian Psi, U_B Psi or
    # B Psi (formed by eda_bhalf_apply on the GPU side, by the oracle's
    # circulant on the other), with q - 1 power passes.  Eigenvalues within
    # the oracle's own sensitivity to a 1e-15 perturbation of Phi; for q = 1
    # also Y = A Phi itself
    spec = S.spec_small(300, 16, 21, every_var=2, every_step=2, length_scale=8.0, seed=7)
    spec = replace(spec, k=15)
    taps, xb, y = problem(spec)
    traj, d, b = oracle_setup(spec, taps, xb, y)
    apply_ctrl = _ctrl_apply(spec, traj, taps)
    rng = np.random.default_rng(100 + q)
    psi = rng.standard_normal((spec.ell, spec.n))  # rows = columns of Psi
    phi_o = psi.copy()
    for _ in range({"psi": 0, "ub_psi": 1, "b_psi": 2}[kind]):
        phi_o = O.bhalf_apply(phi_o, taps)
    _, D, info = O.nystrom(apply_ctrl, phi_o.T, spec.k, q=q)
    _, Dp, _ = O.nystrom(apply_ctrl, phi_o.T * (1 + 1e-15 * rng.standard_normal(phi_o.T.shape)), spec.k, q=q)
    sens = np.abs(Dp - D) / np.maximum(D, 1e-300)
    with make(spec, taps) as h:
        h.eda_set_trajectory(xb, y)
        phi_g = psi.copy()
        for _ in range({"psi": 0, "ub_psi": 1, "b_psi": 2}[kind]):
            tmp = np.zeros_like(phi_g)
            h.eda_bhalf_apply(phi_g, tmp)
            phi_g = tmp
        assert rel(phi_g, phi_o) < 1e-13
        Yg = np.zeros((spec.ell, spec.n))
        h.eda_sketch(phi_g, q, Yg)
        if q == 1:
            assert rel(Yg, info["Y"].T) < 1e-11
        ev = np.zeros(spec.k)
        h.eda_build_lmp(ev)
        path, rank, _ = h.eda_lmp_info()
        top = D > 1e-10 * D[0]  # modes above the sketch's rounding floor
        err = np.abs(ev - 1 - D) / (1 + D)
        assert (err[top] <= np.maximum(1e-9, 100 * sens[top])).all(), (kind, q, path, err.max())
