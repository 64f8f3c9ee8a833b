"""The LMP outside the fused PCG kernels, through the C ABI: eda_lmp_apply
of P_theta, U_theta and U_theta^{-1} (Section 3.1, Eq. (lmp)) on CUDA cores
and on tensor cores (split-BF16, FP32 accumulation) against the oracle; the
split-preconditioner PCG against the oracle's; the tensor-core LMP inside a
solve."""
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


def oracle_coefs(D, theta_mode, theta_given):
    th = O.theta_value(theta_mode, D, theta_given)
    c = O.lmp_coeffs(D, th)
    s = O.lmp_split_coeffs(D, th)
    return c, s, 1.0 / (1.0 + s) - 1.0


# (n, members, ell = k): ragged n, members beyond one 16-wide MMA tile and
# beyond one 256-member group, k not a multiple of 16
CASES = [(40, 11, 10), (997, 21, 13), (4096, 51, 49), (1024, 257, 31)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,M,k", CASES, ids=lambda v: str(v))
def test_lmp_apply_matches_the_oracle(n, M, k, precision):
    spec = S.spec_small(n, 6, M, every_var=2, every_step=2, length_scale=4.0, seed=21)
    spec = replace(spec, ell=k, k=k, spinup=50)
    taps = O.bhalf_taps(n, 4.0, 1.0)
    # an orthonormal S and descending eigenvalues, loaded with eda_set_lmp
    rng = np.random.default_rng(n + k)
    Sk, _ = np.linalg.qr(rng.standard_normal((n, k)))
    D = np.sort(rng.uniform(10.0, 1e4, k))[::-1]
    R = rng.standard_normal((M, n))
    c, s, sinv = oracle_coefs(D, spec.theta_mode, spec.theta)
    prec = P.EDA_FP64 if precision == "fp64" else P.EDA_MIXED
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    with P.Handle.from_spec(spec, taps, precision=prec) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_set_lmp(np.ascontiguousarray(Sk.T), 1 + D)
        for which, coef in ((0, c), (1, s), (2, sinv)):
            ref = O.lmp_apply(Sk, coef, R)
            corr = np.linalg.norm(ref - R, axis=1)
            for kind in (0, 1):
                Z = np.zeros_like(R)
                h.eda_lmp_apply(R, Z, which=which, kind=kind)
                err = np.linalg.norm(Z - ref, axis=1) / corr
                # FP64: rounding; FP32 S and arithmetic: 1e-6; split-BF16:
                # 16 significant bits per operand, FP32 accumulation
                bound = 1e-4 if kind == 1 else (1e-12 if precision == "fp64" else 1e-5)
                assert err.max() < bound, (which, kind, err.max())
        # in place (Z = R) gives the same
        Z = R.copy()
        h.eda_lmp_apply(Z, Z, which=0, kind=1)
        assert (np.linalg.norm(Z - O.lmp_apply(Sk, c, R), axis=1) / np.linalg.norm(R, axis=1)).max() < 1e-4


def test_split_preconditioner_matches_the_oracle():
    # equal iteration counts, one preconditioner (the oracle's S and
    # eigenvalues) on both sides; the split iterates x = U y equal the PCG
    # iterates with P_theta (the oracle's pin), so both oracle runs are the
    # reference here
    spec = S.spec_tiny(seed=14)
    taps, xb, y = problem(spec)
    ref = O.eda_pipeline(spec, xb, y, taps, tol=0, maxit=1, fixed_iters=1)
    traj, b, Sk, D = ref["traj"], ref["b"], ref["S"], ref["D"]
    c, s, _ = oracle_coefs(D, spec.theta_mode, spec.theta)
    hv = lambda V: O.hvp(spec, traj, V, taps)
    K = 6
    osp = O.pcg_split(hv, b, Sk, s, tol=0, maxit=K, fixed_iters=K)
    opc = O.pcg(hv, b, lambda R: O.lmp_apply(Sk, c, R), tol=0, maxit=K, fixed_iters=K)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_set_lmp(np.ascontiguousarray(Sk.T), 1 + D)
        dz = np.zeros_like(b)
        cost = np.zeros((spec.n_members, K + 1))
        it = np.zeros(spec.n_members, np.int32)
        h.eda_solve(dz, tol=0.0, maxit=K, split=True, cost_out=cost, iters_out=it)
        assert (it == K).all()
        assert rowrel(dz, osp["x"]).max() < 1e-10
        assert rowrel(dz, opc["x"]).max() < 1e-10
        Jo = np.array(osp["J"])
        assert np.abs(cost - Jo).max() <= 1e-10 * np.abs(Jo).max()
        # tolerance-stopped, then the certified bound of the mapped solution
        exact = O.eda_pipeline(spec, xb, y, taps, tol=1e-13, maxit=300)["x"]
        eb = np.zeros(spec.n_members)
        st = np.zeros(spec.n_members, np.int32)
        h.eda_solve(dz, tol=1e-8, maxit=300, split=True, err_bound_out=eb, status_out=st)
        assert (st == P.EDA_CONVERGED).all()
        assert (rowrel(dz, exact) <= eb * (1 + 1e-6) + 1e-13).all()
        # the split-BF16 LMP is refused there (its error would meet H's
        # leading eigenvalues between the two applications of U)
        with pytest.raises(P.EdaError) as e:
            h.eda_solve(dz, tol=1e-8, maxit=300, split=True, lmp_kind=1)
        assert e.value.code == P.EDA_ERR_INVALID


def test_tensor_core_lmp_in_the_mixed_solve():
    # the batched-workload shape at reduced size: the split-BF16 LMP
    # preconditions as well as the FP32 one (iteration counts within a few
    # percent) and the certified error stop holds
    spec = S.spec_small(1024, 16, 21, every_var=2, every_step=2, length_scale=8.0, seed=15)
    spec = replace(spec, ell=20, k=19)
    taps, xb, y = problem(spec)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_sketch()
        h.eda_build_lmp()
        out = {}
        for kind in (0, 1):
            dz = np.zeros((spec.n_members, spec.n))
            it = np.zeros(spec.n_members, np.int32)
            eb = np.zeros(spec.n_members)
            st = np.zeros(spec.n_members, np.int32)
            h.eda_solve(dz, tol=1e-6, err_tol=1e-6, maxit=20000, lmp_kind=kind, iters_out=it, err_bound_out=eb,
                        status_out=st)
            assert (st == P.EDA_CONVERGED).all() and (eb <= 1e-6).all()
            out[kind] = (dz, it)
        print("iterations: FP32 LMP %s, split-BF16 LMP %s" % (out[0][1].sum(), out[1][1].sum()))
        assert out[1][1].sum() <= 1.1 * out[0][1].sum()
        assert rowrel(out[1][0], out[0][0]).max() < 4e-6
