"""The learned warm start's hand-written kernels against the FP64 oracle of
the network (same BF16-rounded weights): loss, gradients, inference and one
AdamW step; and the end-to-end use as PCG initial iterate."""
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


@pytest.mark.parametrize("hidden,n", [(8, 96), (64, 128), (5, 37)])
def test_loss_gradient_and_inference_match_oracle(hidden, n):
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
