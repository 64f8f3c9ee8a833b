"""Writes oracle_pcg_iters_n4096.json: PCG iterations to relative residual
1e-6 of the FP64 oracle on the n=4096, 64-step, 51-member workload (seed 0),
for a sample of members (the control and one perturbed member), with the
Gamma-sketch LMP.  Calls only the oracle (several minutes on one core).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import eda_synth as S  # noqa: E402
import oracle as O  # noqa: E402

MEMBERS = [0, 7]


def main():
    spec = S.spec_batched(seed=0)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    traj = O.member_trajectories(spec, xb)
    b = O.rhs(spec, traj, O.innovations(spec, traj, y), taps)
    ctrl = traj[0:1]

    def apply_ctrl(block):
        tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
        return O.apply_A(spec, tr, block.T.copy(), taps).T

    Sk, D, _ = O.nystrom(apply_ctrl, O.gamma(b)[:, : spec.ell], spec.k)
    c = O.lmp_coeffs(D, O.theta_value(spec.theta_mode, D, spec.theta))
    t0 = time.time()
    res = O.pcg(lambda V: O.hvp(spec, traj[MEMBERS], V, taps), b[MEMBERS],
                lambda R: O.lmp_apply(Sk, c, R), tol=1e-6, maxit=10000)
    out = {"workload": spec.name, "seed": 0, "members": MEMBERS, "tol": 1e-6,
           "iters": [int(i) for i in res["iters"]], "relres": [float(r) for r in res["relres"]],
           "status": [int(s) for s in res["status"]], "lambda_max_A": float(D[0]),
           "lambda_k_A": float(D[-1]), "seconds": time.time() - t0}
    with open(os.path.join(HERE, "oracle_pcg_iters_n4096.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
