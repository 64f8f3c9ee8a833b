"""FP64 CPU oracle of the learned warm start (test infrastructure only).

Not a method of the paper: a small periodic 1-D convolutional network that
maps (member right-hand side b_j, control solution dz_0) to a guess of the
member solution dz_j, used only as the initial iterate of the PCG of
Section 2.3 (which then runs to the same tolerance).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module; it shares no code with the CUDA path.

Definition (the reading this package uses):
* inputs X = [b_j / s_b, dz_0 / s_z] (2 channels, length n, periodic), s_b and
  s_z the root-mean-square of b and dz_0 over the training set;
* layers l = 1..4: conv with kernel 5 centred (tap t reads position i + t - 2
  mod n) plus bias; GELU (0.5 x (1 + erf(x / sqrt 2))) after layers 1-3;
  channels 2 -> H -> H -> H -> 1;
* guess dz_j = dz_0 + s_z * out;
* loss = mean over samples and positions of (out + (dz_0 - dz_j) / s_z)^2;
* weights are kept in FP32 and used rounded to BF16 (round to nearest even of
  the FP32 value) in every product; activations and accumulation are exact
  here (FP64);
* AdamW (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay).

Parity: pinned in tests/test_oracle_warmstart.py by central finite
differences of the loss, translation equivariance, and a delta-kernel
identity.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

KSIZE = 5


def bf16_round(a):
    """Round FP64 values to FP32, then to BF16 (round to nearest, ties to
    even) by clearing the low 16 bits of the FP32 pattern; returns FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(hidden):
    return [(hidden, 2), (hidden, hidden), (hidden, hidden), (1, hidden)]


def num_params(hidden):
    return sum(co * ci * KSIZE + co for co, ci in layer_shapes(hidden))


def unflatten(theta, hidden):
    """Flat parameter vector -> [(W (co, ci, K), b (co,)), ...] in layer order."""
    out, o = [], 0
    for co, ci in layer_shapes(hidden):
        W = theta[o: o + co * ci * KSIZE].reshape(co, ci, KSIZE)
        o += co * ci * KSIZE
        b = theta[o: o + co]
        o += co
        out.append((W, b))
    return out


def init_params(hidden, eta):
    """He-scaled weights from standard-normal draws eta (one per parameter;
    biases start at zero)."""
    theta = np.zeros(num_params(hidden))
    o = 0
    for co, ci in layer_shapes(hidden):
        nw = co * ci * KSIZE
        theta[o: o + nw] = eta[o: o + nw] * np.sqrt(2.0 / (ci * KSIZE))
        o += nw + co
    return theta


def conv(x, W, b):
    """Periodic 'same' conv: out[s, o, i] = b[o] + sum_{c,t} W[o,c,t] x[s,c,i+t-2]."""
    out = np.zeros((x.shape[0], W.shape[0], x.shape[2]))
    for t in range(KSIZE):
        xs = np.roll(x, -(t - KSIZE // 2), axis=2)       # xs[..., i] = x[..., i + t - 2]
        out += np.einsum("oc,sci->soi", W[:, :, t], xs)
    return out + b[None, :, None]


def conv_grads(x, W, g):
    """Gradients of sum(g * conv(x, W, b)) w.r.t. x, W and b."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t in range(KSIZE):
        sh = t - KSIZE // 2
        xs = np.roll(x, -sh, axis=2)
        gW[:, :, t] = np.einsum("soi,sci->oc", g, xs)
        gx += np.roll(np.einsum("oc,soi->sci", W[:, :, t], g), sh, axis=2)
    return gx, gW, g.sum(axis=(0, 2))


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def features(rhs, ctrl, s_b, s_z):
    return np.stack([rhs / s_b, ctrl / s_z], axis=1)


def forward(theta, hidden, X):
    """Returns (out (S, n), cache)."""
    layers = unflatten(theta, hidden)
    acts, pres = [X], []
    h = X
    for li, (W, b) in enumerate(layers):
        z = conv(h, bf16_round(W), b)
        pres.append(z)
        h = gelu(z) if li < 3 else z
        acts.append(h)
    return h[:, 0, :], (acts, pres)


def loss_and_grad(theta, hidden, rhs, ctrl, sol, s_b, s_z):
    """Mean loss and its gradient w.r.t. the flat parameters (the gradient of
    the products taken at the BF16-rounded weights)."""
    X = features(rhs, ctrl, s_b, s_z)
    out, (acts, pres) = forward(theta, hidden, X)
    target = (sol - ctrl) / s_z
    diff = out - target
    m = diff.size
    loss = float(np.sum(diff * diff) / m)
    g = (2.0 / m) * diff[:, None, :]
    layers = unflatten(theta, hidden)
    grads = []
    for li in range(3, -1, -1):
        W, b = layers[li]
        if li < 3:
            g = g * gelu_grad(pres[li])
        gx, gW, gb = conv_grads(acts[li], bf16_round(W), g)
        grads.append((gW, gb))
        g = gx
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return loss, np.concatenate(flat)


def guess(theta, hidden, rhs, ctrl, s_b, s_z):
    out, _ = forward(theta, hidden, features(rhs, ctrl, s_b, s_z))
    return ctrl + s_z * out


def adamw_step(theta, grad, m, v, t, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW update (t counts from 1); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v
