"""Seeded synthetic inputs for the Lorenz-96 ensemble-of-4D-Var workloads.

This module holds ONLY random draws and integer structure (problem sizes,
observation patterns, per-observation error variances).  It contains none of
the method's arithmetic: no model step, no covariance square root, no
linear algebra.  Both the CPU oracle (through the tests) and the CUDA path
(through the tests and the benchmark) take their inputs from here, so that
parity never depends on two random number generators agreeing.

Workloads (Section 4 of the paper sets the experiment up as an identical twin
with the Lorenz-96 model; the sizes below are the batched workloads this
package is measured on):

* ``tiny``    : n=40, 20-step window, obs every 2nd variable every 4th step,
                sigma_o=1, length scale 2, 10 members + control, k=ell=10.
* ``batched`` : n=4096, 64-step window, obs every 2nd variable every 2nd step,
                sigma_o=1, length scale 8, 50 members + control, ell=50, k=49.
* ``uneven``  : 256 independent problems, n log-uniform in [40, 8192], window
                log-uniform in [8, 128], members uniform in [10, 80], obs
                density uniform in [0.25, 0.5] (a seeded random subset that
                is the same at every obs step, obs every 2nd step), length
                scale uniform in [2, 16], k = members - 1.
* ``scale``   : n=65536, 96-step window, obs every 2nd variable every 2nd
                step, length scale 8, 80 members + control, ell=80, k=79,
                trajectory checkpoints every 8 steps.
* ``warm``    : n=1024, 32-step window, obs every 2nd variable every 2nd
                step, length scale 4, 256 members + control.
* ``paper``   : the size of the paper's own experiment (Section 4): n=1500,
                10-step window, fifty variables (every 30th) observed at
                three steps (4, 7, 10), sigma_o=0.05, sigma_b=0.8, length
                scale 6 (the Daley length of its diffusion B), 20 members +
                control, ell=k=20.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

THETA_GIVEN = 0
THETA_LAMBDA_K = 1
THETA_MID = 2


@dataclass
class Spec:
    """One EDA problem: sizes, observation network and error scales."""

    n: int
    nsteps: int
    obs_steps: np.ndarray          # int32, sorted, each in [0, nsteps]
    obs_ptr: np.ndarray            # int32, len(obs_steps)+1 (CSR)
    obs_idx: np.ndarray            # int32, variable indices, sorted per step
    sigma_o: float
    sigma_b: float
    length_scale: float
    n_members: int                 # L + 1 (member 0 is the control)
    ell: int
    k: int
    F: float = 8.0
    dt: float = 0.025
    theta_mode: int = THETA_MID
    theta: float = 1.0
    spinup: int = 1000
    spin_sigma: float = 0.1        # N(0, 0.01) read as a variance
    ckpt_every: int = 0
    seed: int = 0
    name: str = ""

    @property
    def p(self) -> int:
        return int(self.obs_ptr[-1])

    @property
    def rinv(self) -> np.ndarray:
        """Diagonal of R^{-1}, one entry per observation (R = sigma_o^2 I)."""
        return np.full(self.p, 1.0 / (self.sigma_o * self.sigma_o), dtype=np.float64)


@dataclass
class Draws:
    """Standard-normal draws of one twin experiment."""

    eta_spin: np.ndarray   # (n,)      spin-up noise
    eta_b: np.ndarray      # (L+1, n)  row 0: control background error
    eta_o: np.ndarray      # (L+1, p)  row 0: truth observation error


def regular_obs(n: int, nsteps: int, every_var: int, every_step: int):
    """Every ``every_var``-th variable at steps every_step, 2*every_step, ...

    Step 0 (the start of the window) carries no observation.
    """
    steps = np.arange(every_step, nsteps + 1, every_step, dtype=np.int32)
    idx1 = np.arange(0, n, every_var, dtype=np.int32)
    ptr = np.arange(len(steps) + 1, dtype=np.int32) * len(idx1)
    idx = np.tile(idx1, len(steps)).astype(np.int32)
    return steps, ptr.astype(np.int32), idx


def subset_obs(n: int, nsteps: int, density: float, every_step: int, rng):
    """A seeded random sorted subset of variables, the same at every obs step."""
    m = max(1, int(round(density * n)))
    idx1 = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    steps = np.arange(every_step, nsteps + 1, every_step, dtype=np.int32)
    if len(steps) == 0:
        steps = np.array([nsteps], dtype=np.int32)
    ptr = (np.arange(len(steps) + 1) * m).astype(np.int32)
    idx = np.tile(idx1, len(steps)).astype(np.int32)
    return steps, ptr, idx


def spec_tiny(seed: int = 0) -> Spec:
    steps, ptr, idx = regular_obs(40, 20, 2, 4)
    return Spec(n=40, nsteps=20, obs_steps=steps, obs_ptr=ptr, obs_idx=idx,
                sigma_o=1.0, sigma_b=1.0, length_scale=2.0, n_members=11,
                ell=10, k=10, seed=seed, name="l96_n40_w20_m11")


def spec_batched(seed: int = 0) -> Spec:
    steps, ptr, idx = regular_obs(4096, 64, 2, 2)
    return Spec(n=4096, nsteps=64, obs_steps=steps, obs_ptr=ptr, obs_idx=idx,
                sigma_o=1.0, sigma_b=1.0, length_scale=8.0, n_members=51,
                ell=50, k=49, seed=seed, name="l96_n4096_w64_m51")


def spec_scale(seed: int = 0) -> Spec:
    steps, ptr, idx = regular_obs(65536, 96, 2, 2)
    return Spec(n=65536, nsteps=96, obs_steps=steps, obs_ptr=ptr, obs_idx=idx,
                sigma_o=1.0, sigma_b=1.0, length_scale=8.0, n_members=81,
                ell=80, k=79, ckpt_every=8, seed=seed, name="l96_n65536_w96_m81")


def spec_warm(seed: int = 0, members: int = 256) -> Spec:
    steps, ptr, idx = regular_obs(1024, 32, 2, 2)
    return Spec(n=1024, nsteps=32, obs_steps=steps, obs_ptr=ptr, obs_idx=idx,
                sigma_o=1.0, sigma_b=1.0, length_scale=4.0, n_members=members + 1,
                ell=min(members, 32), k=min(members, 32) - 1, seed=seed,
                name="l96_n1024_w32_m%d" % (members + 1))


def spec_small(n: int, nsteps: int, members: int, every_var: int = 2, every_step: int = 2,
               length_scale: float = 2.0, ell: Optional[int] = None, k: Optional[int] = None,
               sigma_o: float = 1.0, sigma_b: float = 1.0, seed: int = 0) -> Spec:
    """A free-size problem with a regular observation network (tests)."""
    steps, ptr, idx = regular_obs(n, nsteps, every_var, every_step)
    ell = members - 1 if ell is None else ell
    k = ell if k is None else k
    return Spec(n=n, nsteps=nsteps, obs_steps=steps, obs_ptr=ptr, obs_idx=idx,
                sigma_o=sigma_o, sigma_b=sigma_b, length_scale=length_scale,
                n_members=members, ell=ell, k=k, seed=seed,
                name="l96_n%d_w%d_m%d" % (n, nsteps, members))


def specs_uneven(count: int = 256, seed: int = 0, n_range=(40, 8192), w_range=(8, 128),
                 m_range=(10, 80)) -> List[Spec]:
    """``count`` independent problems of uneven size, drawn from ``seed``."""
    rng = np.random.default_rng([seed, 0x0E7E])
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        nsteps = int(round(np.exp(rng.uniform(np.log(w_range[0]), np.log(w_range[1])))))
        members = int(rng.integers(m_range[0], m_range[1] + 1))
        density = float(rng.uniform(0.25, 0.5))
        lb = float(rng.uniform(2.0, 16.0))
        steps, ptr, idx = subset_obs(n, nsteps, density, 2, rng)
        # k = members - 1 from an ell = members sketch; a sketch cannot have
        # more columns than the state has variables, so ell <= n
        ell = min(members, n)
        out.append(Spec(n=n, nsteps=nsteps, obs_steps=steps, obs_ptr=ptr, obs_idx=idx,
                        sigma_o=1.0, sigma_b=1.0, length_scale=lb,
                        n_members=members + 1, ell=ell, k=ell - 1,
                        seed=seed * 100003 + i, name="uneven_%d" % i))
    return out


def draws(spec: Spec, seed: Optional[int] = None) -> Draws:
    """Standard-normal draws for one twin experiment of ``spec``."""
    s = spec.seed if seed is None else seed
    rng = np.random.default_rng([s, spec.n, spec.nsteps, spec.n_members])
    eta_spin = rng.standard_normal(spec.n)
    eta_b = rng.standard_normal((spec.n_members, spec.n))
    eta_o = rng.standard_normal((spec.n_members, spec.p))
    return Draws(eta_spin=eta_spin, eta_b=eta_b, eta_o=eta_o)


def gaussian_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """A standard Gaussian matrix (sketches, test vectors), row-major (rows, cols)."""
    return np.random.default_rng([seed, rows, cols, 0x5EED]).standard_normal((rows, cols))


def spec_paper(seed: int = 0, k: int = 20) -> Spec:
    n, N = 1500, 10
    steps = np.array([4, 7, 10], dtype=np.int32)
    idx1 = np.arange(0, n, n // 50, dtype=np.int32)
    ptr = (np.arange(len(steps) + 1) * len(idx1)).astype(np.int32)
    return Spec(n=n, nsteps=N, obs_steps=steps, obs_ptr=ptr, obs_idx=np.tile(idx1, len(steps)),
                sigma_o=0.05, sigma_b=0.8, length_scale=6.0, n_members=21, ell=20, k=k,
                seed=seed, name="l96_n1500_w10_m21")


def ensemble_draws(spec: Spec, control_seed: int, member_seed: int) -> Draws:
    """Draws whose truth and control member come from ``control_seed`` and
    whose perturbed members 1..L come from ``member_seed``: one twin
    experiment (one control Hessian) under many ensemble realisations."""
    base = draws(spec, control_seed)
    mem = draws(spec, member_seed)
    eta_b = mem.eta_b.copy()
    eta_o = mem.eta_o.copy()
    eta_b[0] = base.eta_b[0]
    eta_o[0] = base.eta_o[0]
    return Draws(eta_spin=base.eta_spin, eta_b=eta_b, eta_o=eta_o)


def by_name(name: str, seed: int = 0) -> Spec:
    return {"tiny": spec_tiny, "batched": spec_batched, "scale": spec_scale,
            "warm": spec_warm, "paper": spec_paper}[name](seed=seed)
