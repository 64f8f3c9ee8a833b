"""Dependency reach of one RK4 step of the tangent-linear and adjoint
models, which fixes the halo widths of the tiled sweep kernels: a tile that
is refreshed every K steps needs a halo at least as wide as the distance
an error from outside the tile travels inward in K steps.  Measured with
the oracle's exact steps on a periodic state by perturbing everything
outside a tile (state and vector alike) and locating the outputs inside it
that move.

Widths used by the kernels: a warp tile refreshed every step keeps 12
points (16 with 8 values per lane) on each side; a CTA region refreshed
every K steps keeps 8K + 8.
"""
import numpy as np

import oracle as O

F, DT = 8.0, 0.025


def _reach(step, steps=1, n=400, s=150, W=96, seed=0):
    rng = np.random.default_rng(seed)
    x = F + rng.standard_normal(n)
    v = rng.standard_normal(n)
    xs = [x]
    for _ in range(steps):
        xs.append(O.rk4_step(xs[-1], F, DT))
    out_mask = np.ones(n, bool)
    out_mask[s:s + W] = False

    def run(xtraj, vec):
        # tangent linear forward over the steps / adjoint backward over them
        if step is O.tl_step:
            for t in range(steps):
                vec = O.tl_step(xtraj[t], vec, F, DT)
        else:
            for t in reversed(range(steps)):
                vec = O.adj_step(xtraj[t], vec, F, DT)
        return vec

    base = run(xs, v)
    # garbage outside the tile, in the vector and in every trajectory state
    xp = [xx.copy() for xx in xs]
    for xx in xp:
        xx[out_mask] += 3.0 * rng.standard_normal(out_mask.sum())
    vp = v.copy()
    vp[out_mask] += 3.0 * rng.standard_normal(out_mask.sum())
    moved = np.nonzero(np.abs(run(xp, vp) - base)[s:s + W] > 0)[0]
    left = moved[moved < W // 2]
    right = moved[moved >= W // 2]
    return (int(left.max()) + 1 if len(left) else 0, W - int(right.min()) if len(right) else 0)


def test_one_step_reach_fits_the_warp_halo():
    tl = _reach(O.tl_step)
    adj = _reach(O.adj_step)
    # one RK4 step: stencil (j-2, j-1, j+1) applied in four stages
    assert tl == (8, 4), tl
    assert adj == (11, 11), adj
    for C, halo in ((2, 12), (4, 12), (8, 16)):
        assert halo % C == 0 and halo >= max(tl + adj)


def test_k_step_reach_fits_the_cluster_halo():
    for K in (1, 2, 4, 8):
        tl = _reach(O.tl_step, steps=K)
        adj = _reach(O.adj_step, steps=K)
        assert max(tl + adj) <= 8 * K + 8, (K, tl, adj)
