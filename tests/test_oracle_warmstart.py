"""Pins of the warm-start network oracle: finite-difference gradients,
translation equivariance of the periodic convolution, a delta kernel, the
BF16 rounding against its bit-level definition, and an AdamW step against
its closed form."""
import numpy as np
import pytest

import oracle.warmstart as W


def test_bf16_rounding_definition():
    # representable values are unchanged; halfway cases round to even
    assert W.bf16_round(np.array([1.0]))[0] == 1.0
    one_ulp = 2.0 ** -7                      # BF16 spacing at 1
    assert W.bf16_round(np.array([1.0 + one_ulp]))[0] == 1.0 + one_ulp
    assert W.bf16_round(np.array([1.0 + 0.5 * one_ulp]))[0] == 1.0          # tie -> even
    assert W.bf16_round(np.array([1.0 + 1.5 * one_ulp]))[0] == 1.0 + 2 * one_ulp  # tie -> even
    assert W.bf16_round(np.array([1.0 + 0.75 * one_ulp]))[0] == 1.0 + one_ulp
    x = np.random.default_rng(0).standard_normal(1000)
    r = W.bf16_round(x)
    # 8 significant bits: unit roundoff 2^-8
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * 1.0001)


def test_conv_translation_equivariance_and_delta_kernel():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 17))
    Wt = rng.standard_normal((4, 3, 5))
    b = rng.standard_normal(4)
    y = W.conv(x, Wt, b)
    np.testing.assert_allclose(W.conv(np.roll(x, 5, axis=2), Wt, b), np.roll(y, 5, axis=2), atol=1e-12)
    # a delta at tap t copies channel c shifted by t - 2 (periodic wrap)
    D = np.zeros((3, 3, 5))
    for c in range(3):
        D[c, c, 4] = 1.0
    np.testing.assert_allclose(W.conv(x, D, np.zeros(3)), np.roll(x, -2, axis=2), atol=0)


def test_conv_against_direct_loops():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 2, 9))
    Wt = rng.standard_normal((3, 2, 5))
    b = rng.standard_normal(3)
    y = W.conv(x, Wt, b)
    n = 9
    for o in range(3):
        for i in range(n):
            s = b[o] + sum(Wt[o, c, t] * x[0, c, (i + t - 2) % n] for c in range(2) for t in range(5))
            assert abs(s - y[0, o, i]) < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    hidden, n, S = 4, 12, 3
    rhs = rng.standard_normal((S, n))
    ctrl = rng.standard_normal((S, n))
    sol = ctrl + 0.3 * rng.standard_normal((S, n))
    theta = W.init_params(hidden, rng.standard_normal(W.num_params(hidden)))
    # the gradient is taken at the BF16-rounded weights: with every weight
    # pre-rounded, the BF16 network equals an unrounded twin, whose loss is
    # differentiated by central differences

    def loss_exact(th):
        save = W.bf16_round
        try:
            W.bf16_round = lambda a: np.asarray(a, dtype=np.float64)
            return W.loss_and_grad(th, hidden, rhs, ctrl, sol, 1.3, 0.7)[0]
        finally:
            W.bf16_round = save

    th_r = theta.copy()
    # round every weight (biases stay) so that the exact network equals the BF16 one
    layers = W.unflatten(th_r, hidden)
    for Wl, _ in layers:
        Wl[...] = W.bf16_round(Wl)
    loss_r, g_r = W.loss_and_grad(th_r, hidden, rhs, ctrl, sol, 1.3, 0.7)
    assert abs(loss_exact(th_r) - loss_r) < 1e-12
    eps = 1e-6
    idx = rng.choice(len(theta), 40, replace=False)
    for i in idx:
        tp, tm = th_r.copy(), th_r.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (loss_exact(tp) - loss_exact(tm)) / (2 * eps)
        assert abs(fd - g_r[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g_r[i])


def test_adamw_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    grad = np.array([0.3, -0.1, 0.0])
    th, m, v = W.adamw_step(theta, grad, np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.1)
    # first step: m_hat = g, v_hat = g^2, update = lr (sign(g) g/(|g|+eps) + wd theta)
    expect = theta - 0.01 * (grad / (np.abs(grad) + 1e-8) + 0.1 * theta)
    np.testing.assert_allclose(th, expect, atol=1e-15)


def test_training_reduces_loss_on_a_linear_target():
    # a target that is a periodic convolution of the inputs is learnable
    rng = np.random.default_rng(4)
    hidden, n, S = 8, 32, 16
    rhs = rng.standard_normal((S, n))
    ctrl = rng.standard_normal((S, n))
    sol = ctrl + 0.2 * (np.roll(rhs, 1, axis=1) + rhs)
    theta = W.init_params(hidden, rng.standard_normal(W.num_params(hidden)))
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0 = W.loss_and_grad(theta, hidden, rhs, ctrl, sol, 1.0, 1.0)[0]
    for t in range(1, 201):
        loss, g = W.loss_and_grad(theta, hidden, rhs, ctrl, sol, 1.0, 1.0)
        theta, m, v = W.adamw_step(theta, g, m, v, t, lr=3e-3, wd=0.0)
    assert loss < 0.2 * l0


def test_pcg_iterations_fall_only_logarithmically_with_the_guess_error():
    # what any warm start can gain: the oracle's PCG (Section 2.3, with the
    # spectral LMP of Section 3.1) from initial iterates x* + e with smooth
    # errors |e| = eps |x*| needs fewer iterations as eps falls, but only in
    # proportion to log(1 / eps): a guess at 1 % of the solution still needs
    # most of the iterations of a start from zero
    import eda_synth as S
    import oracle as O
    spec = S.spec_small(128, 12, 17, every_var=2, every_step=2, length_scale=4.0, seed=77)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    ref = O.eda_pipeline(spec, xb, y, taps, tol=1e-10, maxit=2000)
    x, b = ref["x"], ref["b"]

    def iters(x0):
        r = O.pcg(lambda V: O.hvp(spec, ref["traj"], V, taps), b, lambda R: O.lmp_apply(ref["S"], ref["c"], R),
                  tol=1e-8, maxit=2000, x0=x0)
        assert (r["status"] == 0).all()
        return int(r["iters"].sum())

    rng = np.random.default_rng(3)
    noise = np.stack([O.bhalf_apply(v, taps) for v in rng.standard_normal(x.shape)])
    noise *= np.linalg.norm(x, axis=1, keepdims=True) / np.linalg.norm(noise, axis=1, keepdims=True)
    n0 = iters(None)
    counts = [iters(x + eps * noise) for eps in (0.5, 0.1, 0.01)]
    assert n0 >= counts[0] >= counts[1] >= counts[2]
    assert counts[2] > 0.5 * n0, (n0, counts)
