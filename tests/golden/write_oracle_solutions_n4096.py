"""Writes oracle_solutions_n4096.npz: reference solutions of the FP64 oracle
on the n=4096, 64-step, 51-member Lorenz-96 workload (seed 0), for a sample
of members, with the Gamma-sketch LMP (Section 3.2.2, Algorithm 1, Section
3.1) and PCG (Section 2.3).  Calls only the oracle (about twenty minutes on
eight cores; one worker process per task, numpy on one thread each).

Stored per sampled member:
  x_tight       the PCG solution at relative residual 1e-13 (or where
                12000 iterations leave it);
  tight_relres  its FP64 true relative residual |b - H x| / |b|;
  tight_bound   |b - H x| / (|x| - |b - H x|), a certified bound on the
                relative error |x - x*| / |x*|: lambda_min(I + A) >= 1
                (Section 2.3) gives |x - x*| <= |b - H x| and
                |x*| >= |x| - |x - x*|;
  iters_1e6     the PCG stopping count at relative residual 1e-6,
  iters_1e6_pert  the same for eight 1e-16 relative perturbations of b
                (how far CG rounding alone moves the count), and
  iters_1e6_pert13  for four 1e-13 relative perturbations (the level at
                which two FP64 implementations of the Hessian product differ).
Also stored: the spun-up truth x^t_0 the twin starts from (so that a caller
can rebuild the same inputs with twin_from_truth, or with a GPU twin started
from it without spin-up), the U_B taps, and the LMP eigenvalues.
"""
import json
import multiprocessing as mp
import os
import sys
import time

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

MEMBERS = [0, 7, 26, 50]
PERT_SEEDS = [1, 2, 3, 4, 5, 6, 7, 8]
PERT13_SEEDS = [11, 12, 13, 14]
TIGHT_TOL, TIGHT_MAXIT = 1e-13, 12000
OUT = os.path.join(HERE, "oracle_solutions_n4096.npz")


def setup():
    import eda_synth as S
    import oracle as O
    spec = S.spec_batched(seed=0)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    xt0, xb, y = O.twin(spec, S.draws(spec), taps)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    ctrl = traj[0:1]

    def apply_ctrl(block):
        tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
        return O.apply_A(spec, tr, block.T.copy(), taps).T

    Sk, D, _ = O.nystrom(apply_ctrl, O.gamma(b)[:, : spec.ell], spec.k)
    c = O.lmp_coeffs(D, O.theta_value(spec.theta_mode, D, spec.theta))
    return spec, taps, xt0, traj, b, Sk, D, c


def task(args):
    import oracle as O
    member, kind, seed = args
    spec, taps, xt0, traj, b, Sk, D, c = setup()
    tr = traj[member:member + 1]
    bm = b[member:member + 1].copy()
    hv = lambda V: O.hvp(spec, tr, V, taps)
    pre = lambda R: O.lmp_apply(Sk, c, R)
    t0 = time.time()
    if kind == "tight":
        res = O.pcg(hv, bm, pre, tol=TIGHT_TOL, maxit=TIGHT_MAXIT)
        x = res["x"][0]
        rt = np.linalg.norm(bm[0] - hv(res["x"])[0])
        xn = np.linalg.norm(x)
        return {"member": member, "kind": kind, "x": x, "iters": int(res["iters"][0]),
                "relres": float(rt / np.linalg.norm(bm[0])), "bound": float(rt / (xn - rt)),
                "seconds": time.time() - t0}
    if seed:
        amp = 1e-13 if seed in PERT13_SEEDS else 1e-16
        bm = bm * (1 + amp * np.random.default_rng(seed).standard_normal(bm.shape))
    res = O.pcg(hv, bm, pre, tol=1e-6, maxit=10000)
    return {"member": member, "kind": kind, "seed": seed, "iters": int(res["iters"][0]),
            "seconds": time.time() - t0}


def main():
    spec, taps, xt0, traj, b, Sk, D, c = setup()
    tasks = [(m, "tight", 0) for m in MEMBERS] + [(m, "tol", s) for m in MEMBERS
                                                  for s in [0] + PERT_SEEDS + PERT13_SEEDS]
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
        res = pool.map(task, tasks, chunksize=1)
    tight = {r["member"]: r for r in res if r["kind"] == "tight"}
    it6 = {(r["member"], r["seed"]): r["iters"] for r in res if r["kind"] == "tol"}
    meta = {"workload": spec.name, "seed": 0, "members": MEMBERS, "tight_tol": TIGHT_TOL,
            "tight_maxit": TIGHT_MAXIT, "perturbation": "b * (1 + 1e-16 N(0,1)), seeds %s; 1e-13, seeds %s"
            % (PERT_SEEDS, PERT13_SEEDS),
            "seconds": {str(m): tight[m]["seconds"] for m in MEMBERS}}
    np.savez_compressed(
        OUT, members=np.array(MEMBERS, np.int32), xt0=xt0, taps=taps, lmp_eigvals=1.0 + D,
        x_tight=np.stack([tight[m]["x"] for m in MEMBERS]),
        tight_iters=np.array([tight[m]["iters"] for m in MEMBERS], np.int32),
        tight_relres=np.array([tight[m]["relres"] for m in MEMBERS]),
        tight_bound=np.array([tight[m]["bound"] for m in MEMBERS]),
        iters_1e6=np.array([it6[(m, 0)] for m in MEMBERS], np.int32),
        iters_1e6_pert=np.array([[it6[(m, s)] for s in PERT_SEEDS] for m in MEMBERS], np.int32),
        iters_1e6_pert13=np.array([[it6[(m, s)] for s in PERT13_SEEDS] for m in MEMBERS], np.int32),
        meta=np.array(json.dumps(meta)))
    print(json.dumps(meta))
    for m in MEMBERS:
        print(m, tight[m]["iters"], tight[m]["relres"], tight[m]["bound"], it6[(m, 0)],
              [it6[(m, s)] for s in PERT_SEEDS], [it6[(m, s)] for s in PERT13_SEEDS])


if __name__ == "__main__":
    main()
