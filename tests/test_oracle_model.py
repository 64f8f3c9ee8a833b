"""Pins of the oracle's model, tangent linear, adjoint and covariance square
root against things other than the oracle itself (Section 4 model ODE, RK4;
Section 2.1 Jacobian; Section 2.3 control-variable transform)."""
import os

import numpy as np
import pytest

import oracle as O

F, DT = 8.0, 0.025


def test_fixed_point_is_preserved_exactly():
    # f(F * 1) = 0 exactly, so every RK4 stage returns the same state.
    x = np.full(37, F)
    traj = O.trajectory(x, F, DT, 200)
    assert np.array_equal(traj[-1], x)


def paper_tendency_loop(x, F):
    """The paper's ODE with its 1-based indices and explicit boundary values
    X^(-1) = X^(n-1), X^(0) = X^(n), X^(n+1) = X^(1), by plain loops."""
    n = len(x)
    X = {j + 1: x[j] for j in range(n)}
    X[-1] = X[n - 1]
    X[0] = X[n]
    X[n + 1] = X[1]
    return np.array([-X[j - 2] * X[j - 1] + X[j - 1] * X[j + 1] - X[j] + F
                     for j in range(1, n + 1)])


def test_tendency_matches_paper_indexing():
    rng = np.random.default_rng(1)
    for n in (4, 5, 13, 40):
        x = rng.standard_normal(n) * 3 + 2
        np.testing.assert_allclose(O.l96_tendency(x, F), paper_tendency_loop(x, F),
                                   rtol=0, atol=1e-12)


def test_energy_identity():
    # The advection term conserves energy: sum_i x_i (x_{i+1} - x_{i-2}) x_{i-1} = 0,
    # so x . f(x) = -|x|^2 + F sum(x).  A wrong sign or index breaks it.
    rng = np.random.default_rng(2)
    for n in (5, 40, 301):
        x = rng.standard_normal(n) * 4
        lhs = float(np.dot(x, O.l96_tendency(x, F)))
        rhs = -float(np.dot(x, x)) + F * float(x.sum())
        assert abs(lhs - rhs) <= 1e-10 * (1 + abs(rhs))


def test_rk4_local_error_order():
    # One RK4 step against a tight adaptive integrator: local error O(dt^5).
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(3)
    x = F + rng.standard_normal(40)
    x = O.trajectory(x, F, DT, 400)[-1]
    errs = []
    for h in (0.04, 0.02, 0.01):
        ref = solve_ivp(lambda t, y: O.l96_tendency(y, F), (0, h), x, method="DOP853",
                        rtol=1e-13, atol=1e-13).y[:, -1]
        errs.append(np.linalg.norm(O.rk4_step(x, F, h) - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 20 < r1 < 45 and 20 < r2 < 45, (errs, r1, r2)


def test_tangent_linear_taylor():
    rng = np.random.default_rng(4)
    n, N = 40, 20
    x0 = O.trajectory(F + rng.standard_normal(n), F, DT, 300)[-1]
    dx = rng.standard_normal(n)
    traj = O.trajectory(x0, F, DT, N)
    m_dx = dx.copy()
    for t in range(N):
        m_dx = O.tl_step(traj[t], m_dx, F, DT)
    base = traj[-1]
    rem = []
    alphas = [10.0 ** (-e) for e in range(1, 6)]
    for a in alphas:
        xa = O.trajectory(x0 + a * dx, F, DT, N)[-1]
        xh = O.trajectory(x0 + 0.5 * a * dx, F, DT, N)[-1]
        ra = np.linalg.norm(xa - base - a * m_dx)
        rh = np.linalg.norm(xh - base - 0.5 * a * m_dx)
        rem.append(ra / rh)
    # second-order remainder: halving alpha divides it by 4
    for r in rem[1:]:
        assert abs(r - 4.0) < 0.1, rem


@pytest.mark.parametrize("n", [5, 8, 40, 97])
def test_adjoint_dot_product(n):
    rng = np.random.default_rng(n)
    x = F + 3 * rng.standard_normal(n)
    d = rng.standard_normal(n)
    w = rng.standard_normal(n)
    lhs = np.dot(O.tl_step(x, d, F, DT), w)
    rhs = np.dot(d, O.adj_step(x, w, F, DT))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # and over a window, through the sweeps used by the Hessian
    traj = O.trajectory(x, F, DT, 15)
    v, u = d.copy(), w.copy()
    for t in range(15):
        v = O.tl_step(traj[t], v, F, DT)
    for t in range(14, -1, -1):
        u = O.adj_step(traj[t], u, F, DT)
    assert abs(np.dot(v, w) - np.dot(d, u)) <= 1e-12 * abs(np.dot(v, w))


def test_jacobian_transpose_entrywise():
    # J^T built from jacT_apply equals the transpose of J built from jac_apply
    rng = np.random.default_rng(7)
    n = 11
    X = rng.standard_normal(n)
    Jm = np.stack([O.jac_apply(X, e) for e in np.eye(n)], axis=1)
    JTm = np.stack([O.jacT_apply(X, e) for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(JTm, Jm.T, atol=1e-14)
    # and J is the derivative of the tendency (central differences)
    eps = 1e-6
    Jfd = np.stack([(O.l96_tendency(X + eps * e, F) - O.l96_tendency(X - eps * e, F)) / (2 * eps)
                    for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(Jm, Jfd, atol=1e-8)


def test_bhalf_taps_closed_form():
    path = os.path.join(os.path.dirname(__file__), "golden", "gaussian_taps_closed_form.txt")
    ref = np.loadtxt(path)
    taps = O.bhalf_taps(256, 2.0, 1.0)
    m = min(len(taps), len(ref))
    np.testing.assert_allclose(taps[:m], ref[:m, 1], rtol=1e-14, atol=0)
    # truncation: taps fall below 1e-17 c_0 beyond w = floor(6.25 L)
    assert len(taps) - 1 == 12
    assert taps[-1] >= 1e-17 * taps[0] and np.exp(-13.0 ** 2 / 4) < 1e-17


@pytest.mark.parametrize("n,L", [(40, 2.0), (128, 8.0), (600, 16.0)])
def test_bhalf_square_is_gaussian_correlation(n, L):
    taps = O.bhalf_taps(n, L, 1.3)
    U = O.bhalf_dense(n, taps)
    assert np.allclose(U, U.T, atol=1e-15)
    B = U @ U
    d = np.arange(n)
    # the correlation on the circle: the Gaussian summed over its periodic images
    target = 1.3 ** 2 * sum(np.exp(-((d + j * n) ** 2) / (2 * L * L)) for j in (-2, -1, 0, 1))
    # first row of B is the correlation function: by Poisson summation the
    # discrete self-convolution of the sampled square root differs from the
    # sampled Gaussian by a relative 2 exp(-pi^2 L^2 / 2) (plus the 1e-17 cut)
    if n > 13 * L:
        bound = 2.5 * np.exp(-np.pi ** 2 * L * L / 2) * 1.3 ** 2 + 1e-14
        np.testing.assert_allclose(B[0], target, rtol=0, atol=bound)
    # always: B is symmetric positive semi-definite
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    assert ev.min() > -1e-12
