"""Test infrastructure (the CPU oracle): a bounded PCG sample of one member,
run in a worker process by the benchmark's all-cores CPU baseline.  Imports
numpy and the oracle only, so that spawned workers start quickly."""
import time

from . import eda_oracle as O


def pcg_member_sample(args):
    """Runs `iters` oracle PCG iterations (Section 2.3) of one member with
    the given LMP and returns the seconds they took.  args = (spec, traj1
    [1, N+1, n], b1 [1, n], S_k [n, k], c [k], taps, iters)."""
    spec, traj1, b1, Sk, c, taps, iters = args
    t0 = time.perf_counter()
    O.pcg(lambda V: O.hvp(spec, traj1, V, taps), b1, lambda R: O.lmp_apply(Sk, c, R),
          tol=0.0, maxit=iters, fixed_iters=iters)
    return time.perf_counter() - t0
