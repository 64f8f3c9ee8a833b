"""The learned warm start's hand-written kernels against the FP64 oracle of
the network (same BF16-rounded weights): loss, gradients, inference and one
AdamW step, on CUDA cores and with the tensor-core convolutions; and the
end-to-end use as PCG initial iterate."""
import numpy as np
import pytest

import eda_synth as S
import oracle as O
import oracle.warmstart as W
from helpers import problem, rowrel

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_23571_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def net_case(hidden=8, n=96, S_=6, seed=0):
    rng = np.random.default_rng(seed)
    rhs = rng.standard_normal((S_, n)) * 3.0
    ctrl = rng.standard_normal((S_, n)) * 0.5
    sol = ctrl + 0.3 * np.roll(rhs, 1, axis=1) / 3.0 + 0.05 * rng.standard_normal((S_, n))
    eta = S.gaussian_matrix(1, W.num_params(hidden), seed + 100)[0]
    theta = W.init_params(hidden, eta)
    # biases nonzero so that they are exercised
    for _, b in W.unflatten(theta, hidden):
        b[...] = 0.1 * rng.standard_normal(b.shape)
    theta = theta.astype(np.float32).astype(np.float64)   # FP32 masters
    return rhs, ctrl, sol, theta


@pytest.mark.parametrize("hidden,n", [(8, 96), (64, 128), (5, 37), (64, 1000)])
def test_loss_gradient_and_inference_match_oracle(hidden, n):
    # hidden = 64 takes the tensor-core convolutions for the 64 -> 64 layers
    # (n = 1000: eight position tiles, the last one ragged)
    rhs, ctrl, sol, theta = net_case(hidden, n)
    sb, sz = 2.9, 0.55
    loss_o, grad_o = W.loss_and_grad(theta, hidden, rhs, ctrl, sol, sb, sz)
    guess_o = W.guess(theta, hidden, rhs, ctrl, sb, sz)
    with P.WarmStart(n, hidden, max_batch=8) as ws:
        ws.eda_ws_set_params(theta.astype(np.float32))
        ws.eda_ws_set_scales(sb, sz)
        loss_g, grad_g = ws.eda_ws_loss_grad(rhs, ctrl, sol)
        out = np.zeros_like(rhs)
        ws.eda_ws_infer(rhs, ctrl, out)
    assert abs(loss_g - loss_o) <= 1e-5 * loss_o
    # FP32 accumulation (atomics in any order) against FP64
    err = np.abs(grad_g - grad_o)
    assert err.max() <= 2e-4 * np.abs(grad_o).max() + 1e-7, err.max()
    assert rowrel(out, guess_o).max() < 1e-5


def test_adamw_step_matches_oracle():
    hidden, n = 8, 64
    rhs, ctrl, sol, theta = net_case(hidden, n, S_=4, seed=3)
    sb, sz = 3.0, 0.5
    loss, g = W.loss_and_grad(theta, hidden, rhs, ctrl, sol, sb, sz)
    th1, _, _ = W.adamw_step(theta, g, np.zeros_like(theta), np.zeros_like(theta), 1, lr=1e-3, wd=0.01)
    with P.WarmStart(n, hidden, max_batch=4) as ws:
        ws.eda_ws_set_params(theta.astype(np.float32))
        ws.eda_ws_set_scales(sb, sz)
        losses = ws.eda_ws_train(rhs, ctrl, sol, epochs=1, batch=4, lr=1e-3, weight_decay=0.01)
        th_g = ws.eda_ws_get_params().astype(np.float64)
    assert abs(losses[0] - loss) <= 1e-5 * loss
    # first AdamW step moves each weight by ~lr * sign(g); the FP32 update
    # agrees with the FP64 one except where |g| is near rounding
    d_o, d_g = th1 - theta, th_g - theta
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    np.testing.assert_allclose(d_g[big], d_o[big], rtol=2e-3, atol=2e-7)


def test_training_learns_a_periodic_convolution():
    hidden, n, S_ = 16, 64, 32
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal((S_, n))
    ctrl = rng.standard_normal((S_, n))
    sol = ctrl + 0.2 * (np.roll(rhs, 1, axis=1) + rhs)
    theta = W.init_params(hidden, S.gaussian_matrix(1, W.num_params(hidden), 7)[0])
    with P.WarmStart(n, hidden, max_batch=32) as ws:
        ws.eda_ws_set_params(theta.astype(np.float32))
        losses = ws.eda_ws_train(rhs, ctrl, sol, epochs=300, batch=32, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0], losses[[0, -1]]


def test_he_initialisation_matches_oracle():
    hidden, n = 16, 48
    with P.WarmStart(n, hidden, max_batch=4) as ws:
        eta = S.gaussian_matrix(1, ws.num_params, 7)[0]
        ws.eda_ws_init(eta)
        got = ws.eda_ws_get_params()
    ref = W.init_params(hidden, eta)
    np.testing.assert_allclose(got, ref.astype(np.float32), rtol=1e-6, atol=0)


def test_warm_start_gain_on_held_out_problems():
    # training triples (member RHS, control solution, member solution) from
    # the plain FP64 solver on small problems, the network trained on the GPU
    # (AdamW, cosine learning-rate schedule), then a held-out problem solved
    # from zero and from the network's guess to the same tolerance: the guess
    # must beat the control solution as a guess, the warm-started solve must
    # need fewer member iterations in all, both solves converge and agree
    # within the residual bound, and the iterations saved are reported
    import torch
    dev = torch.device("cuda:0")
    n, N, members = 256, 16, 64

    def problem_on_gpu(seed):
        spec = S.spec_small(n, N, members + 1, every_var=2, every_step=2, length_scale=4.0, seed=seed)
        taps = P.bhalf_gaussian(n, spec.length_scale, spec.sigma_b)
        h = P.Handle.from_spec(spec, taps, precision=P.EDA_FP64)
        dr = S.draws(spec)
        M = spec.n_members
        xb = torch.empty(M, n, dtype=torch.float64, device=dev)
        y = torch.empty(M, spec.p, dtype=torch.float64, device=dev)
        h.eda_twin(torch.tensor(spec.F + spec.spin_sigma * dr.eta_spin, device=dev), 300,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        b = torch.empty(M, n, dtype=torch.float64, device=dev)
        h.eda_set_trajectory(xb, y, b)
        h.eda_sketch()
        h.eda_build_lmp()
        return h, b

    def solve(h, b, x0=None):
        M = b.shape[0]
        dz = torch.empty_like(b)
        it = np.zeros(M, np.int32)
        rr = np.zeros(M)
        st = np.zeros(M, np.int32)
        h.eda_solve_batch(1e-8, 5000, x0, True, dz, it, rr, st)
        return dz, it, rr, st

    R, C, Z = [], [], []
    for e in range(12):
        h, b = problem_on_gpu(100 + e)
        dz, _, _, st = solve(h, b)
        h.close()
        assert (st == P.EDA_CONVERGED).all()
        R.append(b[1:])
        C.append(dz[0:1].expand(members, -1))
        Z.append(dz[1:])
    R, C, Z = (torch.cat(v).contiguous() for v in (R, C, Z))
    with P.WarmStart(n, 32, max_batch=64) as ws:
        ws.eda_ws_init(S.gaussian_matrix(1, ws.num_params, 5)[0])
        losses = []
        for e in range(30):
            order = np.random.default_rng(e).permutation(R.shape[0]).astype(np.int32)
            lr = 0.5 * 2e-3 * (1 + np.cos(np.pi * e / 30))
            losses.append(ws.eda_ws_train(R, C, Z, epochs=1, batch=64, lr=lr, order=order)[0])
        assert losses[-1] < losses[0]
        h, b = problem_on_gpu(900)
        dz0, it0, rr0, st0 = solve(h, b)
        ctrl = dz0[0:1].expand(members, -1).contiguous()
        guess = torch.empty(members, n, dtype=torch.float64, device=dev)
        ws.eda_ws_infer(b[1:].contiguous(), ctrl, guess)
        x0 = torch.cat([dz0[0:1], guess]).contiguous()
        dzw, itw, rrw, stw = solve(h, b, x0)
        h.close()
    ref = dz0[1:]
    err_guess = (torch.linalg.norm(guess - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy()
    err_ctrl = (torch.linalg.norm(ctrl - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy()
    print("warm start: guess error median %.3f (control as guess %.3f); member iterations %d -> %d (%.1f %% saved)"
          % (np.median(err_guess), np.median(err_ctrl), it0[1:].sum(), itw[1:].sum(),
             100.0 * (1 - itw[1:].sum() / it0[1:].sum())))
    assert np.median(err_guess) < np.median(err_ctrl)
    assert (st0 == P.EDA_CONVERGED).all() and (stw == P.EDA_CONVERGED).all()
    # CG's count falls only with the logarithm of the initial error (about
    # 1 % here for a guess at 0.6 of the solution), but it must fall
    assert itw[1:].sum() < it0[1:].sum()
    # both solutions are within their residuals of the exact one (lambda_min >= 1)
    bn = torch.linalg.norm(b, dim=1).cpu().numpy()
    diff = torch.linalg.norm(dzw - dz0, dim=1).cpu().numpy()
    assert (diff <= (rr0 + rrw) * bn * (1 + 1e-6) + 1e-12).all()


def test_tensor_core_and_cuda_core_convolutions_agree():
    # the same network and batch with the 64 -> 64 layers on the tensor cores
    # and on CUDA cores (EDA_WS_TC=0): both take FP32 activations times BF16
    # weights with FP32 accumulation, which the tensor cores sum in another
    # order and round differently; held to each other by the bars both keep
    # against the FP64 oracle (measured loss difference 5e-6 relative)
    from helpers import env
    hidden, n = 64, 700
    rhs, ctrl, sol, theta = net_case(hidden, n, S_=5, seed=9)
    res = {}
    for tc in (1, 0):
        with env(EDA_WS_TC=tc):
            with P.WarmStart(n, hidden, max_batch=8) as ws:
                ws.eda_ws_set_params(theta.astype(np.float32))
                ws.eda_ws_set_scales(2.5, 0.6)
                loss, grad = ws.eda_ws_loss_grad(rhs, ctrl, sol)
                out = np.zeros_like(rhs)
                ws.eda_ws_infer(rhs, ctrl, out)
                res[tc] = (loss, grad, out)
    (l1, g1, o1), (l0, g0, o0) = res[1], res[0]
    assert abs(l1 - l0) <= 2e-5 * l0
    assert np.abs(g1 - g0).max() <= 2e-4 * np.abs(g0).max()
    assert rowrel(o1, o0).max() < 2e-5
