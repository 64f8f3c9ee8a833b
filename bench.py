"""Benchmark of the EDA hot path on GB300: member solves/s to relative residual
1e-6 of the plain FP64 GPU path (the headline, at the paper's precision),
beside the mixed-precision and tensor-core-LMP forms at equal certified
accuracy, Hessian-vector products/s, the rooflines of the sweeps, and the CPU
oracle timed beside it.

One step = the whole path on one synthetic EDA of the n=4096, 64-step,
51-member Lorenz-96 workload: nonlinear trajectories, innovations and
right-hand sides of all members, the Gamma sketch of the control Hessian,
the Nystrom factorisation and LMP, and the batched PCG of all 51 members to
relative residual 1e-6.  Every form's solutions are compared with reference
solutions (the FP64 path at relative residual 1e-12, with certified error
bounds) and, on sampled members, with the FP64 oracle's.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank runs an
independent replica on its own GPU (the path has no data exchange between
EDA problems); value = member solves of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

# the CPU oracle baseline reports the threads it uses: one (numpy's BLAS
# pinned to a single thread before numpy loads)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np
from dataclasses import replace

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import eda_synth as S  # noqa: E402

METRIC = "EDA member solves/s to rel-res 1e-6 & Hv products/s vs plain FP64 GPU path"
UNIT = "member solves/s"
TOL = 1e-6
MAXIT = 6000
MAXIT_ERR = 20000  # budget of the certified-error forms (deeper than relres 1e-6)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the scale, uneven-batch and warm-start measurements")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile-case", choices=["fp64", "mixed", "scale", "lmp", "hvp32"], default=None,
                    help="profiling case for ncu: fp64 / mixed: the workload's setup, sketch and LMP, then one "
                         "PCG solve of --profile-iters fixed iterations between cudaProfilerStart/Stop; scale: "
                         "one batched FP32 Hessian product of --profile-members members of the scale workload "
                         "(its multi-launch chain) in that range; lmp: the LMP apply on CUDA and tensor cores "
                         "timed at the batched and the scale sizes, the batched size's tensor-core apply in that "
                         "range; hvp32: the batched workload's FP32 member Hessian products through eda_hvp (one "
                         "column per member, each on its own trajectory), three of them in that range; prints one "
                         "line")
    ap.add_argument("--profile-iters", type=int, default=20)
    ap.add_argument("--profile-members", type=int, default=9)
    ap.add_argument("--profile-ckpt", type=int, default=0,
                    help="scale profiling case: the trajectory checkpointed every this many steps (0: stored)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t, device):
    """The largest of every rank's t (the job's time: the slowest replica)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_value(members, steps, world, t_max):
    """Whole-job member solves/s of `world` independent replicas, each solving
    `members` members per step for `steps` steps, over the slowest time."""
    return world * members * steps / t_max


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the samples go to a temporary file that the summary reads back
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="eda_clocks_%d_" % gpu_index, suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def persist_traffic_per_launch(plan, dtype, cols_per_launch):
    """DRAM bytes (read + write) per launch of the persistent PCG kernel:
    the committed ncu summary's bytes per member-iteration (a 20-iteration
    capture of the same kernel and workload; the per-iteration traffic of the
    steady state) times the member-iterations a launch of the timed steps ran,
    or None when the code or the tiling differs from the captured one."""
    path = PERSIST_PROFILE[dtype]
    if plan is None or not os.path.exists(path) or cols_per_launch <= 0:
        return None
    txt = open(path).read()
    m_sha = re.search(r"sweep\.cu code sha256: ([0-9a-f]{64})", txt)
    m_b = re.search(r"dram bytes per member-iteration \(read \+ write\): ([0-9.eE+]+)", txt)
    m_p = re.search(r"captured plan: kind=(\S+) ctas_per_vector=(\d+) threads=(\d+) C=(\d+) K=(\d+)", txt)
    if not (m_sha and m_b and m_p) or code_sha256(SWEEP_SRC) != m_sha.group(1):
        return None
    cap = (m_p.group(1),) + tuple(int(v) for v in m_p.groups()[1:])
    if cap != (plan["kind"], plan["ctas_per_vector"], plan["threads"], plan["C"], plan["K"]):
        return None
    return float(m_b.group(1)) * cols_per_launch


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


SWEEP_SRC = os.path.join(ROOT, "paper_2605_23571_gb300", "csrc", "sweep.cu")
SWEEP_PROFILE = os.path.join(ROOT, "profiles", "sweep_kernel_f32_member_hvp_l96_n4096_w64_m51.md")
PERSIST_PROFILE = {"double": os.path.join(ROOT, "profiles", "pcg_persist_kernel_f64_l96_n4096_w64_m51.md"),
                   "float": os.path.join(ROOT, "profiles", "pcg_persist_kernel_f32_l96_n4096_w64_m51.md")}


def persist_kernel_name(plan, dtype="double", tails=()):
    """The persistent PCG kernel a cluster tiling launches (EDA_PERSIST unset
    or 1), or None for tilings the per-iteration launches serve; tails: the
    (level, plan) tilings of the convergence tail (eda_tail_plans)."""
    if plan["kind"] != "cluster" or os.environ.get("EDA_PERSIST", "1") == "0":
        return None
    tail = "".join("; at <= %d active members %d CTAs x %d threads, refresh every %d"
                   % (lv, t["ctas_per_vector"], t["threads"], t["K"]) for lv, t in tails)
    return ("pcg_persist_kernel<%s,%d> (one cluster of %d CTAs x %d threads per member, halo refresh every %d "
            "steps%s: the member's sweeps, CG updates, LMP and stopping test, one launch per phase of the solve)"
            % (dtype, plan["C"], plan["ctas_per_vector"], plan["threads"], plan["K"], tail))


def sweep_kernel_name(plan, dtype="float"):
    """The sweep kernel a tiling from eda_sweep_plan launches, with its shape."""
    if plan["kind"] == "warp":
        return "wsweep_kernel<%s,%d> (warp-tiled: %d CTAs per vector x %d threads, halo refresh every %d steps)" % (
            dtype, plan["C"], plan["ctas_per_vector"], plan["threads"], plan["K"])
    if plan["kind"] == "multi-launch":
        return "sweep_kernel<%s,%d> (multi-launch: %d tiles per vector x %d threads, %d steps per launch)" % (
            dtype, plan["C"], plan["ctas_per_vector"], plan["threads"], plan["K"])
    return "sweep_kernel<%s,%d> (clusters of %d CTAs x %d threads, halo refresh every %d steps)" % (
        dtype, plan["C"], plan["ctas_per_vector"], plan["threads"], plan["K"])


def code_sha256(path):
    """sha256 of a CUDA source with its comments and blank lines removed (the
    code the counters were taken on; comment edits do not change it)."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()


def sweep_traffic_per_launch(plan=None, profile=None):
    """DRAM bytes (read + write) per launch of a member-HVP sweep from its
    committed ncu summary, or None when the sweep's code has changed since
    those counters were taken, when the tiling in use (plan, from
    eda_sweep_plan) is not the captured one, or there is no summary."""
    profile = SWEEP_PROFILE if profile is None else profile
    if not os.path.exists(profile):
        return None
    txt = open(profile).read()
    m_sha = re.search(r"sweep\.cu code sha256: ([0-9a-f]{64})", txt)
    m_b = re.search(r"dram bytes per launch \(read \+ write\): ([0-9.eE+]+)", txt)
    m_p = re.search(r"captured plan: kind=(\S+) ctas_per_vector=(\d+) threads=(\d+) C=(\d+) K=(\d+)", txt)
    if not (m_sha and m_b and m_p):
        return None
    if code_sha256(SWEEP_SRC) != m_sha.group(1):
        return None
    if plan is not None:
        cap = (m_p.group(1),) + tuple(int(v) for v in m_p.groups()[1:])
        if cap != (plan["kind"], plan["ctas_per_vector"], plan["threads"], plan["C"], plan["K"]):
            return None
    return float(m_b.group(1))


# ---------------------------------------------------------------- workload
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_solutions_n4096.npz")


def workload(seed):
    spec = S.spec_batched(seed=seed)
    dr = S.draws(spec)
    return spec, dr


def golden(spec, seed):
    """The oracle's reference solutions of this workload (seed 0 only), with
    the spun-up truth they start from, or None (data file written by
    tests/golden/write_oracle_solutions_n4096.py; nothing is executed)."""
    if seed != 0 or not os.path.exists(GOLDEN):
        return None
    G = dict(np.load(GOLDEN))
    if G["xt0"].shape != (spec.n,):
        return None
    return G


def workload_config(spec, world):
    """The config object of both arms' JSON lines."""
    return {"workload": spec.name, "n": spec.n, "window": spec.nsteps, "members": spec.n_members,
            "ell": spec.ell, "k": spec.k, "obs_per_step": int(spec.p // len(spec.obs_steps)),
            "obs_steps": int(len(spec.obs_steps)), "tol": TOL, "precision": "fp64",
            "l2": "flushed between timed steps (512 MB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def cpu_oracle_parallel(spec, traj, b, Sk, c, taps, cores, sample_iters):
    """The oracle's PCG on `cores` members at once, one spawned worker process
    per member (members are independent; each worker runs numpy on one
    thread): seconds for one iteration of all of them together."""
    import multiprocessing as mp
    from oracle.sample import pcg_member_sample
    m = max(1, min(cores, spec.n_members))
    ctx = mp.get_context("spawn")
    with ctx.Pool(m) as pool:  # leaving the block terminates the workers
        # bounded waits: a stuck pool raises instead of holding the benchmark
        pool.map_async(pcg_member_sample, [(spec, traj[:1], b[:1], Sk, c, taps, 1)] * m).get(timeout=300)
        t0 = time.perf_counter()
        pool.map_async(pcg_member_sample, [(spec, traj[j:j + 1], b[j:j + 1], Sk, c, taps, sample_iters)
                                           for j in range(m)]).get(timeout=300)
        wall = time.perf_counter() - t0
    return m, wall / sample_iters


def cpu_oracle_step(spec, xb, y, taps, iters_per_member, sample_iters=30, cores=1):
    """The oracle on a bounded sample of one step: setup, RHS, Gamma sketch and
    LMP of every member, then ``sample_iters`` PCG iterations of one member;
    the full step is extrapolated with ``iters_per_member`` (the iteration
    count each member needs to reach the tolerance).  With cores > 1 the PCG
    sample also runs on that many members at once in worker processes, and
    the all-cores step is extrapolated from it (members spread evenly over
    the workers; the setup part stays as measured on one core)."""
    import oracle as O
    t0 = time.perf_counter()
    traj = O.member_trajectories(spec, xb)
    d = O.innovations(spec, traj, y)
    b = O.rhs(spec, traj, d, taps)
    ctrl = traj[0:1]

    def apply_ctrl(block):
        tr = np.broadcast_to(ctrl, (block.shape[1],) + ctrl.shape[1:])
        return O.apply_A(spec, tr, block.T.copy(), taps).T

    Sk, D, info = O.nystrom(apply_ctrl, O.gamma(b)[:, : spec.ell], spec.k)
    theta = O.theta_value(spec.theta_mode, D[: info["rank"]], spec.theta)
    c = O.lmp_coeffs(D, theta)
    t1 = time.perf_counter()
    O.pcg(lambda V: O.hvp(spec, traj[:1], V, taps), b[:1], lambda R: O.lmp_apply(Sk, c, R),
          tol=0.0, maxit=sample_iters, fixed_iters=sample_iters)
    t2 = time.perf_counter()
    t_iter = (t2 - t1) / sample_iters
    total_iters = float(np.sum(iters_per_member))
    full = (t1 - t0) + t_iter * total_iters
    out = {"t_setup_sketch_lmp_s": t1 - t0, "t_iter_s": t_iter, "t_full_step_s": full, "t_sample_s": t2 - t0,
           "sample": "numpy FP64 oracle: setup, RHS, Gamma sketch and LMP of all %d members "
                     "(%.1f s) plus %d PCG iterations of one member (%.3f s each), extrapolated "
                     "to the %d PCG iterations (summed over members) the step needs"
                     % (spec.n_members, t1 - t0, sample_iters, t_iter, int(total_iters))}
    if cores > 1:
        try:
            m, t_round = cpu_oracle_parallel(spec, traj, b, Sk, c, taps, cores, sample_iters)
        except Exception as e:  # the one-thread baseline stands without it
            out["all_cores"] = {"unavailable": "worker processes failed: %s" % str(e)[:200]}
            return out
        out["all_cores"] = {
            "cores": m, "t_full_step_s": (t1 - t0) + t_round * total_iters / m,
            "sample": "the same setup, then %d PCG iterations of %d members at once in %d spawned "
                      "worker processes (%.3f s per iteration of all of them), extrapolated with the "
                      "members spread evenly over the workers" % (sample_iters, m, m, t_round)}
    return out


def oracle_iters_per_member(spec):
    """PCG iterations per member of the oracle on this workload: the mean of
    its stopping counts at 1e-6 on the sampled members (committed fixture
    written from the oracle by tests/golden/write_oracle_solutions_n4096.py),
    for every member.  Both CPU baselines extrapolate with these."""
    d = np.load(GOLDEN)
    return np.full(spec.n_members, float(np.mean(d["iters_1e6"])))


def run_reference(args):
    """The oracle (the only reference: the paper ships no code) on the host."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    spec, dr = workload(args.seed)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, dr, taps)
    iters = oracle_iters_per_member(spec)
    for _ in range(args.warmup):
        cpu_oracle_step(spec, xb, y, taps, iters, sample_iters=5)
    times, sampled = [], []
    r = None
    for _ in range(args.steps):
        r = cpu_oracle_step(spec, xb, y, taps, iters)
        times.append(r["t_full_step_s"])
        sampled.append(r["t_sample_s"])
    t = float(np.sum(times))
    value = spec.n_members * args.steps / t
    # ms_per_step: what each timed step took (its bounded sample); the value
    # rests on the full step extrapolated from it
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(sampled)),
            "ms_per_full_step_extrapolated": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(spec, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": r["sample"] + " (iteration counts: the oracle's own on sampled members, "
                                       "tests/golden/oracle_solutions_n4096.npz)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# algorithmic FP32 operations per element-step of one member-column HVP: the
# tangent-linear RK4 step (57) and the adjoint step with its stage
# recomputation (60), counting each multiply and add (Lorenz-96 stencils of
# the oracle's tl_step / adj_step)
FLOPS_PER_ELEMENT_STEP = 117
# the same for the FP64 sweep that reads the stored RK4 stage states: the
# tangent-linear step (37) and the adjoint step (42) without recomputation
FLOPS_PER_ELEMENT_STEP_STORED = 79


def fp64_peak_tflops(sm_mhz):
    """FP64 FMA peak of a GB300 derived from its nominal 1.25 TFLOP/s:
    152 SMs x 2 FP64 FMA per clock x 2 flops."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak of a GB300: 152 SMs x 128 lanes x 2 flops per cycle."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def forms_scale(P, dev, hbm_peak):
    """Scale workload (n=65536, 96-step window, 81 members): the batched
    member HVP in FP32 and FP64 on the tuned tiling, with its HBM and FP32
    ALU roofline fractions and the FP32 sweep's error against FP64."""
    import torch
    spec = S.spec_scale(seed=0)
    spec.ckpt_every = 0
    taps = P.bhalf_gaussian(spec.n, spec.length_scale, spec.sigma_b)
    dr = S.draws(spec)
    M, n, p, N = spec.n_members, spec.n, spec.p, spec.nsteps
    hg = P.Handle.from_spec(spec, taps, precision=P.EDA_FP64)
    xb = torch.empty(M, n, dtype=torch.float64, device=dev)
    y = torch.empty(M, p, dtype=torch.float64, device=dev)
    hg.eda_twin(torch.tensor(spec.F + spec.spin_sigma * dr.eta_spin, device=dev), spec.spinup,
                torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
    hg.close()
    cols = torch.arange(M, dtype=torch.int32, device=dev)
    V = torch.tensor(S.gaussian_matrix(M, n, 31), device=dev)
    out = {}
    HV = {}
    for prec, key in ((P.EDA_MIXED, "fp32"), (P.EDA_FP64, "fp64")):
        with P.Handle.from_spec(spec, taps, precision=prec) as h:
            h.eda_set_trajectory(xb, y)
            h.eda_autotune(0)
            ms = h.eda_time_hvp_sweep(reps=5 if key == "fp32" else 2, fp64=(key == "fp64"))
            out["ms_per_batched_hvp_" + key] = ms
            hv = torch.empty_like(V)
            h.eda_hvp(cols, V, hv, True)
            HV[key] = hv
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(HV["fp32"] - HV["fp64"], dim=1) / torch.linalg.norm(HV["fp64"], dim=1)).max().item()
    ms32 = out["ms_per_batched_hvp_fp32"]
    bytes_launch = M * 4 * n * (2 * N + 2)
    flops_launch = FLOPS_PER_ELEMENT_STEP * M * n * N
    gbs = bytes_launch / (ms32 / 1e3) / 1e9
    tfl = flops_launch / (ms32 / 1e3) / 1e12
    peak_alu = fp32_peak_tflops(2070.0)
    out.update({
        "workload": spec.name, "columns": M, "trajectory_bytes_fp32": M * (N + 1) * n * 4,
        "hv_per_s_fp32": M / (ms32 / 1e3),
        "roofline_hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                         "bytes_per_launch": bytes_launch},
        "roofline_alu": {"achieved": tfl, "peak": peak_alu, "unit": "TFLOP/s", "frac": tfl / peak_alu,
                         "flops_per_launch": flops_launch,
                         "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
        "fp32_vs_fp64_hvp_relerr_max": rel,
    })
    # the precision-at-scale configuration as specified: the trajectory
    # checkpointed every 8 steps (13 stored states per member instead of 97),
    # FP32 sweeps recomputing each segment on the chip, the 79-mode LMP
    # applied as split-BF16 tensor-core products, FP64 CG with FP64 true
    # residuals; PCG to relative residual 1e-6 within a stated budget
    spec8 = replace(spec, ckpt_every=8)
    budget = 300
    ck = {"ckpt_every": 8, "stored_states_per_member": N // 8 + 1,
          "trajectory_bytes_fp64": M * (N // 8 + 1) * n * 8, "iteration_budget_per_member": budget}
    with P.Handle.from_spec(spec8, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(xb, y)
        ck["ms_per_batched_hvp_fp64"] = h.eda_time_hvp_sweep(reps=2, fp64=True)
    with P.Handle.from_spec(spec8, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_autotune(2)
        ck["ms_per_batched_hvp_fp32"] = h.eda_time_hvp_sweep(reps=5)
        hv = torch.empty_like(V)
        h.eda_hvp(cols, V, hv, True)
        torch.cuda.synchronize()
        ck["fp32_vs_fp64_hvp_relerr_max"] = (torch.linalg.norm(hv - HV["fp64"], dim=1)
                                             / torch.linalg.norm(HV["fp64"], dim=1)).max().item()
        ev = np.zeros(spec8.k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.eda_sketch()
        h.eda_build_lmp(ev)
        torch.cuda.synchronize()
        ck["ms_sketch_plus_lmp"] = 1e3 * (time.perf_counter() - t0)
        ck["lambda_1_and_k"] = [float(ev[0]), float(ev[-1])]
        dz = torch.empty(M, n, dtype=torch.float64, device=dev)
        it = np.zeros(M, np.int32)
        rr = np.zeros(M)
        eb = np.zeros(M)
        st = np.zeros(M, np.int32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.eda_solve(dz, tol=TOL, maxit=budget, lmp_kind=1, iters_out=it, relres_out=rr, err_bound_out=eb,
                    status_out=st)
        torch.cuda.synchronize()
        ck["solve_s"] = time.perf_counter() - t0
        ck.update({"converged": int((st == 0).sum()), "members": M, "iters_median": float(np.median(it)),
                   "true_relres_median": float(np.median(rr)), "true_relres_max": float(rr.max()),
                   "certified_error_bound_median": float(np.median(eb)),
                   "lmp": "79 modes, split-BF16 on tensor cores"})
    out["ckpt8_mixed_tc_solve"] = ck
    return out


def forms_tiny(P, dev, problems=100):
    """The tiny FP64 workload (n=40, 20-step window, 10 members + control,
    k=10, PCG to 1e-6 within 100 iterations): the latency of one problem's
    setup + sketch + LMP + solve on one handle, and the throughput of 100
    seeded problems as one group."""
    import torch
    specs = [S.spec_tiny(seed=s_) for s_ in range(problems)]
    hs, xbs, ys = [], [], []
    for s_ in specs:
        taps = P.bhalf_gaussian(s_.n, s_.length_scale, s_.sigma_b)
        h = P.Handle.from_spec(s_, taps, precision=P.EDA_FP64)
        dr = S.draws(s_)
        xb = torch.empty(s_.n_members, s_.n, dtype=torch.float64, device=dev)
        y = torch.empty(s_.n_members, s_.p, dtype=torch.float64, device=dev)
        h.eda_twin(torch.tensor(s_.F + s_.spin_sigma * dr.eta_spin, device=dev), s_.spinup,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        hs.append(h)
        xbs.append(xb)
        ys.append(y)
    M = specs[0].n_members
    dz = torch.empty(M, specs[0].n, dtype=torch.float64, device=dev)
    def one_problem(h, xb, y):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.eda_set_trajectory(xb, y)
        h.eda_sketch()
        h.eda_build_lmp()
        h.eda_solve_batch(TOL, 100, None, True, dz)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # one problem end to end: on a handle's first use (its lazily allocated
    # buffers included), and again on a handle in use (a cycling assimilation)
    lat = [one_problem(hs[rep], xbs[rep], ys[rep]) for rep in range(6)]
    lat_warm = [one_problem(hs[0], xbs[rep], ys[rep]) for rep in range(6)]
    with P.Group(hs) as g:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.eda_group_set_trajectories(xbs, ys)
        g.eda_group_sketch()
        g.eda_group_build_lmp()
        T = g.total_members
        it = np.zeros(T, np.int32)
        st = np.zeros(T, np.int32)
        g.eda_group_solve(TOL, 100, True, None, it, None, st)
        torch.cuda.synchronize()
        tg = time.perf_counter() - t0
    for h in hs:
        h.close()
    return {"workload": "l96_n40_w20_m11 x %d seeds" % problems, "precision": "fp64",
            "us_per_problem_single_handle": 1e6 * float(np.median(lat[1:])),
            "us_per_problem_handle_in_use": 1e6 * float(np.median(lat_warm[1:])),
            "group_member_solves_per_s": int((st == 0).sum()) / tg, "group_seconds": tg,
            "group_converged": int((st == 0).sum()), "group_member_solves": T,
            "iters_median": float(np.median(it)), "iters_max": int(it.max())}


def forms_uneven(P, dev, count=256, maxit=3000):
    """Uneven batch: 256 independent problems in one group (mixed precision,
    autotuned tiling, the PCG as one persistent work-queue launch per tile
    shape), each member with a budget of maxit iterations.  Reports, per
    problem with members that miss the budget, its size, window and the
    count that missed."""
    import torch
    specs = S.specs_uneven(count, seed=0)
    hs, xbs, ys = [], [], []
    for s_ in specs:
        taps = P.bhalf_gaussian(s_.n, s_.length_scale, s_.sigma_b)
        h = P.Handle.from_spec(s_, taps, precision=P.EDA_MIXED)
        dr = S.draws(s_)
        xb = torch.empty(s_.n_members, s_.n, dtype=torch.float64, device=dev)
        y = torch.empty(s_.n_members, s_.p, dtype=torch.float64, device=dev)
        h.eda_twin(torch.tensor(s_.F + s_.spin_sigma * dr.eta_spin, device=dev), s_.spinup,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        hs.append(h)
        xbs.append(xb)
        ys.append(y)
    with P.Group(hs) as g:
        g.eda_group_set_trajectories(xbs, ys)
        g.eda_group_sketch()
        g.eda_group_build_lmp()
        g.eda_group_autotune()
        T = g.total_members
        it = np.zeros(T, np.int32)
        rr = np.zeros(T)
        st = np.zeros(T, np.int32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.eda_group_solve(TOL, maxit, True, None, it, rr, st)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    for h in hs:
        h.close()
    conv = int((st == 0).sum())
    # members of problem i are rows off[i] .. off[i+1] of the group's outputs
    off = np.cumsum([0] + [s_.n_members for s_ in specs])
    missed = []
    for i, s_ in enumerate(specs):
        bad = int((st[off[i]:off[i + 1]] != 0).sum())
        if bad:
            missed.append({"problem": i, "n": s_.n, "window": s_.nsteps, "members": s_.n_members,
                           "missed_budget": bad, "relres_median_missed":
                           float(np.median(rr[off[i]:off[i + 1]][st[off[i]:off[i + 1]] != 0]))})
    return {"workload": "uneven_256_seed0", "problems": count, "member_solves": T, "converged": conv,
            "budget_per_member": maxit, "seconds": t, "converged_solves_per_s": conv / t,
            "iters_median": float(np.median(it)), "iters_p90": float(np.percentile(it, 90)),
            "true_relres_max_converged": float(rr[st == 0].max()) if conv else None,
            "problems_missing_budget": missed,
            "window_of_problems_missing_budget": {"min": min((m["window"] for m in missed), default=None),
                                                  "max": max((m["window"] for m in missed), default=None)},
            "window_all_problems": {"min": int(min(s_.nsteps for s_ in specs)),
                                    "max": int(max(s_.nsteps for s_ in specs))}}


def forms_sketch_study(P, dev, seeds=20, iters=(1, 2, 3, 5, 10, 20, 30)):
    """The paper's experiment at its own size (Section 4: n=1500, 10-step
    window, 50 variables observed at 3 steps, 20 members, ell=20) on the GPU
    path: Algorithm 1 on the control member's Hessian with the five sketch
    matrices Omega = Psi, A Psi (q=2), B Psi, U_B^T Psi and Gamma, and the
    Ritz LMP of ell CG iterations on the control member's Hessian from member
    1's right-hand side, each over `seeds` realisations (Gaussian Psi; ensemble perturbations for Gamma, the
    control member fixed).  Reports the median relative eigenvalue error
    |lambda* - lambda| / lambda* of lambda_i(I + A) against the eigenvalues of
    the dense operator (assembled from n products), the median quadratic-cost
    reduction (J(dz_i) - J*) / (J(0) - J*) of the control member after i PCG
    iterations with each LMP (theta = (lambda_k + 1)/2, k = 20), the same for
    Omega = Gamma with theta in {lambda_k, (lambda_k + 1)/2, 1} and k in {15,
    20}, and the GPU time of sketch + LMP per variant."""
    import torch
    spec0 = S.spec_paper()
    n, M, ell = spec0.n, spec0.n_members, spec0.ell
    taps = P.bhalf_gaussian(n, spec0.length_scale, spec0.sigma_b)

    def twin(h, dr):
        xb = torch.empty(M, n, dtype=torch.float64, device=dev)
        y = torch.empty(M, spec0.p, dtype=torch.float64, device=dev)
        h.eda_twin(torch.tensor(spec0.F + spec0.spin_sigma * dr.eta_spin, device=dev), spec0.spinup,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        return xb, y

    configs = {"k20_mid": (20, S.THETA_MID), "k20_lamk": (20, S.THETA_LAMBDA_K), "k20_one": (20, S.THETA_GIVEN),
               "k15_mid": (15, S.THETA_MID), "k15_lamk": (15, S.THETA_LAMBDA_K), "k15_one": (15, S.THETA_GIVEN)}
    hs = {name: P.Handle.from_spec(replace(spec0, k=k, theta_mode=tm, theta=1.0), taps, precision=P.EDA_FP64)
          for name, (k, tm) in configs.items()}
    h = hs["k20_mid"]
    # the control member's operator I + A, assembled from n products
    xb, y = twin(h, S.ensemble_draws(spec0, 0, 0))
    rhs = torch.empty(M, n, dtype=torch.float64, device=dev)
    h.eda_set_trajectory(xb, y, rhs)
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    Hd = torch.empty_like(eye)
    h.eda_hvp(torch.zeros(n, dtype=torch.int32, device=dev), eye, Hd, True)
    H = Hd.cpu().numpy()
    H = 0.5 * (H + H.T)
    lam_star = np.linalg.eigvalsh(H)[::-1][:ell]
    b0 = rhs[0].cpu().numpy()
    x_star = np.linalg.solve(H, b0)
    J_star = -0.5 * float(b0 @ x_star)

    def cost_reduction(hh, use_lmp):
        dz = torch.empty(M, n, dtype=torch.float64, device=dev)
        out = []
        for i in iters:
            hh.eda_solve_batch(0.0, i, None, use_lmp, dz)
            z = dz[0].cpu().numpy()
            J = 0.5 * float(z @ H @ z) - float(b0 @ z)
            out.append((J - J_star) / (0.0 - J_star))
        return out

    # ritz_cg: the spectral LMP from the Ritz pairs of ell CG iterations on
    # the control member's Hessian, run from another right-hand side (member
    # 1's b, standing in for an earlier CG run of the same system)
    variants = ("psi", "a_psi", "b_psi", "ubt_psi", "gamma", "ritz_cg")
    err = {v: [] for v in variants}
    red = {v: [] for v in variants}
    ms = {v: [] for v in variants}
    sens = {name: [] for name in configs}
    red_none = []
    for seed in range(seeds):
        xb, y = twin(h, S.ensemble_draws(spec0, 0, 1000 + seed))
        rhs_s = torch.empty(M, n, dtype=torch.float64, device=dev)
        for hh in hs.values():
            hh.eda_set_trajectory(xb, y, rhs_s)
        psi = torch.tensor(S.gaussian_matrix(ell, n, 2000 + seed), device=dev)
        ub = torch.empty_like(psi)
        h.eda_bhalf_apply(psi, ub)
        bpsi = torch.empty_like(psi)
        h.eda_bhalf_apply(ub, bpsi)
        phis = {"psi": (psi, 1), "a_psi": (psi, 2), "b_psi": (bpsi, 1), "ubt_psi": (ub, 1), "gamma": (None, 1),
                "ritz_cg": (None, 0)}
        for v in variants:
            phi, q = phis[v]
            ev = np.zeros(spec0.k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if v == "ritz_cg":
                ev[:] = h.eda_ritz_lmp(member=0, iters=ell, b=rhs_s[1])[:spec0.k]
            else:
                h.eda_sketch(phi, q)
                h.eda_build_lmp(ev)
            torch.cuda.synchronize()
            ms[v].append(1e3 * (time.perf_counter() - t0))
            err[v].append(np.abs(lam_star - ev) / lam_star)
            red[v].append(cost_reduction(h, True))
        for name, hh in hs.items():
            hh.eda_sketch()
            hh.eda_build_lmp()
            sens[name].append(cost_reduction(hh, True))
        red_none.append(cost_reduction(h, False))
    for hh in hs.values():
        hh.close()
    pick = (0, 4, 9, 14, 19)
    med = lambda a: np.median(np.asarray(a), axis=0)
    return {
        "workload": "%s, %d realisations" % (spec0.name, seeds),
        "lambda_star_1_5_10_15_20": [float(lam_star[i]) for i in pick],
        "median_rel_eig_error_modes_1_5_10_15_20": {v: [float(med(err[v])[i]) for i in pick] for v in variants},
        "pcg_iters": list(iters),
        "median_cost_reduction": dict({v: [float(x) for x in med(red[v])] for v in variants},
                                      no_lmp=[float(x) for x in med(red_none)]),
        "gamma_theta_k_cost_reduction": {name: [float(x) for x in med(sens[name])] for name in configs},
        "ms_sketch_plus_lmp": {v: float(np.median(ms[v])) for v in variants},
    }


def forms_warm(P, dev, train_edas=80, test_edas=2, epochs=30, hidden=64, lr0=2e-3):
    """Learned warm start (n=1024, 32-step window, 256 members): training
    triples (member RHS, control solution, member solution) from the plain
    solver, the network trained on the GPU by the library's kernels (AdamW,
    a cosine learning-rate schedule over the epochs), then held-out problems
    solved from zero and from the network's guess to the same tolerance, on
    the FP64 path and in the mixed form (solve time only: the guess's
    inference is reported beside it)."""
    import torch
    n = 1024

    def setup(seed, prec):
        spec = S.spec_warm(seed=seed)
        M = spec.n_members
        taps = P.bhalf_gaussian(n, spec.length_scale, spec.sigma_b)
        h = P.Handle.from_spec(spec, taps, precision=prec)
        dr = S.draws(spec)
        xb = torch.empty(M, n, dtype=torch.float64, device=dev)
        y = torch.empty(M, spec.p, dtype=torch.float64, device=dev)
        h.eda_twin(torch.tensor(spec.F + spec.spin_sigma * dr.eta_spin, device=dev), spec.spinup,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        b = torch.empty(M, n, dtype=torch.float64, device=dev)
        h.eda_set_trajectory(xb, y, b)
        h.eda_sketch()
        h.eda_build_lmp()
        return h, b

    def solve(h, M, x0=None):
        dz = torch.empty(M, n, dtype=torch.float64, device=dev)
        it = torch.empty(M, dtype=torch.int32, device=dev)
        st = torch.empty(M, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.eda_solve_batch(TOL, 20000, x0, True, dz, it, None, st)
        torch.cuda.synchronize()
        return dz, it.cpu().numpy(), st.cpu().numpy(), time.perf_counter() - t0

    R, Cc, Z = [], [], []
    t0 = time.perf_counter()
    for e in range(train_edas):
        h, b = setup(10 ** 6 + e, P.EDA_MIXED)
        dz, _, _, _ = solve(h, b.shape[0])
        R.append(b[1:])
        Cc.append(dz[0:1].expand(dz.shape[0] - 1, -1))
        Z.append(dz[1:])
        h.close()
    R, Cc, Z = (torch.cat(v).contiguous() for v in (R, Cc, Z))
    t_data = time.perf_counter() - t0
    ws = P.WarmStart(n, hidden, max_batch=64)
    ws.eda_ws_init(S.gaussian_matrix(1, ws.num_params, 42)[0])
    t0 = time.perf_counter()
    losses = []
    for e in range(epochs):
        lr = 0.5 * lr0 * (1.0 + np.cos(np.pi * e / epochs))
        order = np.random.default_rng(e).permutation(R.shape[0]).astype(np.int32)
        losses.append(ws.eda_ws_train(R, Cc, Z, epochs=1, batch=64, lr=lr, weight_decay=0.0, order=order))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    losses = np.concatenate(losses)
    out = {"workload": "l96_n1024_w32_m257", "training_triples": int(R.shape[0]), "data_s": t_data,
           "train_s": t_train, "epochs": epochs, "lr": "cosine from %g" % lr0,
           "loss_first_last": [float(losses[0]), float(losses[-1])]}
    for prec, key in ((P.EDA_FP64, "fp64"), (P.EDA_MIXED, "mixed")):
        zero_it, warm_it, ctrl_it, zero_t, warm_t, inf_t, ok = 0, 0, 0, 0.0, 0.0, 0.0, True
        zero_max, warm_max = [], []
        eg, ec = [], []
        for e in range(test_edas):
            h, b = setup(2 * 10 ** 6 + e, prec)
            M = b.shape[0]
            solve(h, M)  # warm-up of this handle's kernels
            dz, it0, st0, tz = solve(h, M)
            guess = torch.empty(M - 1, n, dtype=torch.float64, device=dev)
            ctrl = dz[0:1].expand(M - 1, -1).contiguous()
            torch.cuda.synchronize()
            ti = time.perf_counter()
            ws.eda_ws_infer(b[1:].contiguous(), ctrl, guess)
            torch.cuda.synchronize()
            inf_t += time.perf_counter() - ti
            ref = dz[1:]
            eg.append((torch.linalg.norm(guess - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy())
            ec.append((torch.linalg.norm(ctrl - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy())
            _, itw, stw, tw = solve(h, M, x0=torch.cat([dz[0:1], guess]).contiguous())
            _, itc, _, _ = solve(h, M, x0=torch.cat([dz[0:1], ctrl]).contiguous())
            h.close()
            zero_it += int(it0[1:].sum())
            warm_it += int(itw[1:].sum())
            ctrl_it += int(itc[1:].sum())
            zero_max.append(int(it0[1:].max()))
            warm_max.append(int(itw[1:].max()))
            zero_t += tz
            warm_t += tw
            ok = ok and bool((st0 == 0).all() and (stw == 0).all())
        members = test_edas * 256
        out[key] = {"held_out_members": members, "iters_zero_start": zero_it, "iters_warm_start": warm_it,
                    "iters_control_solution_as_guess": ctrl_it,
                    "iterations_saved_frac": 1.0 - warm_it / max(1, zero_it),
                    "iters_max_zero_per_problem": zero_max, "iters_max_warm_per_problem": warm_max,
                    "guess_rel_err_median": float(np.median(np.concatenate(eg))),
                    "control_solution_rel_err_median": float(np.median(np.concatenate(ec))),
                    "solves_per_s_zero": members / zero_t, "solves_per_s_warm": members / warm_t,
                    "inference_ms_per_problem": 1e3 * inf_t / test_edas, "all_converged": ok}
    ws.close()
    return out


def rel_err(a, ref):
    """Per-member relative error |a - ref| / |ref|."""
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


def err_summary(dz, ref, ref_bound, G=None):
    """Errors of one form's solutions: against the FP64 GPU reference (every
    member; its own certified bound stated), and against the oracle's
    reference solutions of the sampled members when they exist."""
    e = rel_err(dz, ref)
    out = {"vs_fp64_reference": {"max": float(e.max()), "median": float(np.median(e)),
                                 "members_above_1e-6": int((e > 1e-6).sum()),
                                 "reference_certified_bound_max": float(np.max(ref_bound))}}
    if G is not None:
        mem = G["members"]
        eo = rel_err(dz[mem], G["x_tight"])
        out["vs_oracle"] = {"members": [int(m) for m in mem], "rel_err": [float(v) for v in eo],
                            "oracle_certified_bound": [float(v) for v in G["tight_bound"]]}
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2605_23571_gb300 as P
    P.build()
    seed = args.seed + rank
    spec, dr = workload(seed)
    G = golden(spec, seed)
    taps = P.bhalf_gaussian(spec.n, spec.length_scale, spec.sigma_b)
    M, n, p = spec.n_members, spec.n, spec.p
    stream = torch.cuda.current_stream(dev)

    # synthetic identical twin generated on the GPU by the library; with the
    # oracle's reference data for this workload, from the same spun-up truth
    # (so that the oracle's solutions apply to these inputs)
    hgen = P.Handle.from_spec(spec, taps, precision=P.EDA_FP64)
    xb = torch.empty(M, n, dtype=torch.float64, device=dev)
    y = torch.empty(M, p, dtype=torch.float64, device=dev)
    if G is not None:
        x_spin0, spinup = torch.tensor(G["xt0"], device=dev), 0
    else:
        x_spin0, spinup = torch.tensor(spec.F + spec.spin_sigma * dr.eta_spin, device=dev), spec.spinup
    hgen.eda_twin(x_spin0, spinup, torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
    hgen.close()

    dz = torch.empty(M, n, dtype=torch.float64, device=dev)
    iters = torch.empty(M, dtype=torch.int32, device=dev)
    relres = torch.empty(M, dtype=torch.float64, device=dev)
    status = torch.empty(M, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    def step(h, xb_, y_, dz_, it_, rr_, st_, marks=None, etol=0.0, tol=TOL, lmp_kind=0, maxit=MAXIT):
        # marks: events recorded between the phases (setup | sketch + LMP | solve)
        h.eda_set_trajectory(xb_, y_)
        if marks:
            marks[0].record(stream)
        h.eda_sketch()
        h.eda_build_lmp()
        if marks:
            marks[1].record(stream)
        if etol > 0.0 or lmp_kind:
            h.eda_solve(dz_, tol=tol, err_tol=etol, maxit=maxit, lmp_kind=lmp_kind, iters_out=it_,
                        relres_out=rr_, status_out=st_)
        else:
            h.eda_solve_batch(tol, maxit, None, True, dz_, it_, rr_, st_)

    phase_ms = {}

    def timed_steps(h, k, warm, key, **kw):
        for _ in range(warm):
            step(h, xb, y, dz, iters, relres, status, **kw)
        torch.cuda.synchronize()
        tot = 0.0
        its = []
        ph = np.zeros(3)
        for _ in range(k):
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            marks = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e0.record(stream)
            step(h, xb, y, dz, iters, relres, status, marks, **kw)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
            ph += [e0.elapsed_time(marks[0]), marks[0].elapsed_time(marks[1]), marks[1].elapsed_time(e1)]
            its.append(iters.cpu().numpy().copy())
        phase_ms[key] = ph / max(1, k)
        return tot, its

    h64 = P.Handle.from_spec(spec, taps, precision=P.EDA_FP64)
    hm = P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED)
    # setup (untimed): the autotuner picks the sweep tilings on this workload
    h64.eda_set_trajectory(xb, y)
    h64.eda_autotune(0)
    hm.eda_set_trajectory(xb, y)
    hm.eda_autotune(0)
    plan64 = h64.eda_sweep_plan(fp64=True)
    plan32 = hm.eda_sweep_plan(fp64=False)
    tails64 = h64.eda_tail_plans(fp64=True)
    tails32 = hm.eda_tail_plans(fp64=False)

    # ---- timed region (headline: the plain FP64 GPU path at the paper's precision)
    for _ in range(args.warmup):
        step(h64, xb, y, dz, iters, relres, status)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = P.kernel_launches()
    h64.eda_trace(True, every=8)  # one sweep in 8 event-timed inside the timed steps (roofline)
    torch.cuda.profiler.start()  # ncu --profile-from-start off captures from here
    with Clocks(local) as clk:
        t64, its64 = timed_steps(h64, args.steps, 0, "fp64")
    torch.cuda.profiler.stop()
    h64.eda_trace(False)
    launches = P.kernel_launches() - launches0
    sw_calls, sw_cols, sw_ms = h64.eda_trace_read(fp64=True)
    st64 = status.cpu().numpy()
    rr64 = relres.cpu().numpy()
    dz64 = dz.cpu().numpy()
    if world > 1:
        t64 = max_over_ranks(t64, dev)
    value = replica_value(M, args.steps, world, t64)

    # ---- reference solutions (untimed): the FP64 path solved to relative
    # residual 1e-12, each member with its certified error bound
    dz_ref = torch.empty_like(dz)
    eb_ref = np.zeros(M)
    it_ref = np.zeros(M, np.int32)
    h64.eda_solve(dz_ref, tol=1e-12, maxit=12000, err_bound_out=eb_ref, iters_out=it_ref)
    ref = dz_ref.cpu().numpy()

    # ---- the forms beside the headline, on the same workload
    k_m = max(2, min(args.steps, 5))
    forms_solve = {}

    def form(key, h, k, warm, **kw):
        t, its = timed_steps(h, k, warm, key, **kw)
        sol = dz.cpu().numpy()
        its_c = np.concatenate(its)
        out = {"value": M * k / t, "unit": UNIT, "ms_per_step": 1e3 * t / k, "steps": k,
               "iters_min": int(its_c.min()), "iters_median": float(np.median(its_c)), "iters_max": int(its_c.max()),
               "all_converged": bool((status.cpu().numpy() == 0).all()),
               "error": err_summary(sol, ref, eb_ref, G)}
        out.update({"criterion": {"tol_relres": kw.get("tol", TOL), "err_tol": kw.get("etol", 0.0),
                                  "maxit": kw.get("maxit", MAXIT)},
                    "lmp": "split-BF16 tensor cores" if kw.get("lmp_kind", 0) else "CUDA cores"})
        forms_solve[key] = out
        return out

    # mixed precision at the headline's criterion, its sweeps traced for the
    # FP32 roofline
    hm.eda_trace(True, every=8)
    tmix, itsmix = timed_steps(hm, k_m, 2, "mixed")
    hm.eda_trace(False)
    sw32_calls, sw32_cols, sw32_ms = hm.eda_trace_read(fp64=False)
    mix_sol = dz.cpu().numpy()
    its_c = np.concatenate(itsmix)
    forms_solve["mixed_relres_1e-6"] = {
        "value": M * k_m / tmix, "unit": UNIT, "ms_per_step": 1e3 * tmix / k_m, "steps": k_m,
        "iters_min": int(its_c.min()), "iters_median": float(np.median(its_c)), "iters_max": int(its_c.max()),
        "all_converged": bool((status.cpu().numpy() == 0).all()), "true_relres_max": float(relres.cpu().numpy().max()),
        "error": err_summary(mix_sol, ref, eb_ref, G), "criterion": {"tol_relres": TOL, "err_tol": 0.0},
        "lmp": "CUDA cores (FP32)"}
    # equal, certified accuracy: every member stops when its FP64 true
    # residual certifies |dz - dz*| / |dz*| <= 1e-6 (lambda_min(I + A) >= 1)
    f64e = form("fp64_err_1e-6", h64, max(1, min(args.steps, 2)), 0, tol=0.0, etol=1e-6, maxit=MAXIT_ERR)
    form("mixed_err_1e-6", hm, k_m, 1, tol=0.0, etol=1e-6, maxit=MAXIT_ERR)
    form("mixed_tc_lmp_err_1e-6", hm, k_m, 1, tol=0.0, etol=1e-6, lmp_kind=1, maxit=MAXIT_ERR)
    form("mixed_tc_lmp_relres_1e-6", hm, k_m, 1, lmp_kind=1)
    for key in ("mixed_err_1e-6", "mixed_tc_lmp_err_1e-6"):
        forms_solve[key]["speedup_over_fp64_at_equal_accuracy"] = forms_solve[key]["value"] / f64e["value"]
    forms_solve["mixed_relres_1e-6"]["speedup_over_fp64_relres_1e-6"] = (
        forms_solve["mixed_relres_1e-6"]["value"] / (value / world))

    # ---- Hessian-vector products/s and the rooflines of the sweeps
    ms32 = hm.eda_time_hvp_sweep(reps=20)
    ms64 = h64.eda_time_hvp_sweep(reps=3)
    hvps32 = M / (ms32 / 1e3)
    hvps64 = M / (ms64 / 1e3)
    # FP64 sweep: the cluster tiling reads the stored stage states, the
    # warp-tiled one recomputes them
    f64 = FLOPS_PER_ELEMENT_STEP if plan64["kind"] == "warp" else FLOPS_PER_ELEMENT_STEP_STORED
    bytes64_col = 8 * n * (2 * spec.nsteps + 2)
    peak64 = fp64_peak_tflops(2070.0)
    ach64 = f64 * spec.nsteps * n * sw_cols / (sw_ms / 1e3) / 1e12
    hbm_peak, peak_kind = measured_peaks()
    bytes_per_col = 4 * n * (2 * spec.nsteps + 2)
    ach32 = bytes_per_col * sw32_cols / (sw32_ms / 1e3) / 1e9
    if persist_kernel_name(plan64) is not None:
        traffic64 = persist_traffic_per_launch(plan64, "double", sw_cols / max(1, sw_calls))
    else:
        traffic64 = None
    if persist_kernel_name(plan32) is not None:
        traffic32 = persist_traffic_per_launch(plan32, "float", sw32_cols / max(1, sw32_calls))
    else:
        traffic32 = sweep_traffic_per_launch(plan32, SWEEP_PROFILE)

    # ---- end to end through the C ABI with host buffers (headline path)
    xb_h = xb.cpu().pin_memory().numpy()
    y_h = y.cpu().pin_memory().numpy()
    dz_h = torch.empty(M, n, dtype=torch.float64).pin_memory().numpy()
    it_h = torch.empty(M, dtype=torch.int32).pin_memory().numpy()
    rr_h = torch.empty(M, dtype=torch.float64).pin_memory().numpy()
    st_h = torch.empty(M, dtype=torch.int32).pin_memory().numpy()
    k_e2e = max(1, min(args.steps, 3))
    te = 0.0
    for _ in range(k_e2e):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(h64, xb_h, y_h, dz_h, it_h, rr_h, st_h)
        torch.cuda.synchronize()
        te += time.perf_counter() - t0
    e2e = {"value": M * k_e2e / te, "unit": UNIT, "steps": k_e2e,
           "h2d_bytes_per_step": int(xb_h.nbytes + y_h.nbytes),
           "d2h_bytes_per_step": int(dz_h.nbytes + it_h.nbytes + rr_h.nbytes + st_h.nbytes)}

    # ---- CPU oracle baseline (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_step(spec, xb.cpu().numpy(), y.cpu().numpy(), taps, oracle_iters_per_member(spec),
                            cores=os.cpu_count() or 1)
        cpu = {"value": M / r["t_full_step_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": r["sample"] + " (iteration counts: the oracle's own on sampled members, "
                                       "tests/golden/oracle_solutions_n4096.npz, as the reference arm)"}
        if "all_cores" in r:
            ac = r["all_cores"]
            cpu["all_cores"] = ac if "unavailable" in ac else {
                "value": M / ac["t_full_step_s"], "unit": UNIT, "cores": ac["cores"],
                "host_cpus": os.cpu_count(), "sample": ac["sample"]}

    hm.close()
    h64.close()
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:  # single-GPU measurements
        forms = {"tiny": forms_tiny(P, dev), "scale": forms_scale(P, dev, hbm_peak), "uneven": forms_uneven(P, dev),
                 "warm_start": forms_warm(P, dev), "sketch_study": forms_sketch_study(P, dev)}
    if rank == 0:
        its_d = np.concatenate(its64)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t64 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(spec, world),
            "step_ms": {name: {"setup": float(ph[0]), "sketch_lmp": float(ph[1]), "solve": float(ph[2])}
                        for name, ph in phase_ms.items()},
            "solve": {"iters_min": int(its_d.min()), "iters_median": float(np.median(its_d)),
                      "iters_max": int(its_d.max()), "all_converged": bool((st64 == 0).all()),
                      "relres_max": float(rr64.max()), "error": err_summary(dz64, ref, eb_ref, G),
                      "reference": {"what": "FP64 path solved to relative residual 1e-12 (untimed)",
                                    "certified_bound_max": float(eb_ref.max()),
                                    "iters_max": int(it_ref.max())},
                      "inputs": "twin from the oracle's spun-up truth (tests/golden)" if G is not None
                                else "twin spun up on the GPU"},
            "forms_solve": forms_solve,
            "hv_per_s": {"fp64_sweep": hvps64, "fp32_sweep": hvps32,
                         "ms_per_batched_launch_fp64": ms64, "ms_per_batched_launch_fp32": ms32},
            "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                         "frac": ach64 / peak64, "traffic": traffic64,
                         "kernel": (persist_kernel_name(plan64, "double", tails64) or sweep_kernel_name(plan64, "double")
                                    + ": the FP64 Hessian-product sweeps of the timed steps"),
                         "achieved_counts": "algorithmic flops of the sweeps only (79 per element-step) over the "
                                            "whole kernel time (the CG vector work and LMP inside it included)",
                         "flops_per_element_step": f64, "launches_timed": sw_calls, "columns": sw_cols,
                         "ms_per_launch": sw_ms / max(1, sw_calls),
                         "bytes_per_launch": bytes64_col * sw_cols / max(1, sw_calls),
                         "achieved_hbm_gbs": bytes64_col * sw_cols / (sw_ms / 1e3) / 1e9, "hbm_peak": hbm_peak,
                         "peak_kind": "derived from the nominal GB300 FP64 rate: 152 SMs x 2 FP64 FMA/clk x 2 "
                                      "flops x 2070 MHz (no FP64 peak is measured)"},
            "roofline_fp32_sweep": {"bound": "hbm", "achieved": ach32, "peak": hbm_peak, "unit": "GB/s",
                                    "frac": ach32 / hbm_peak, "traffic": traffic32,
                                    "kernel": (persist_kernel_name(plan32, "float", tails32) or sweep_kernel_name(plan32)
                                               + ": the FP32 Hessian-product sweeps of the mixed form's timed steps"),
                                    "launches_timed": sw32_calls, "columns": sw32_cols,
                                    "ms_per_launch": sw32_ms / max(1, sw32_calls),
                                    "bytes_per_launch": bytes_per_col * sw32_cols / max(1, sw32_calls),
                                    "alu_tflops": FLOPS_PER_ELEMENT_STEP * spec.nsteps * n * sw32_cols
                                                  / (sw32_ms / 1e3) / 1e12,
                                    "alu_peak": fp32_peak_tflops(2070.0),
                                    "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs, burst copy); ALU: "
                                                 "152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "forms": forms,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def run_profile_scale(args):
    """The scale workload's batched FP32 Hessian product for a reduced number
    of members (the trajectory still far larger than L2), on the autotuned
    tiling, once inside a profiler range: a small case of the multi-launch
    chain for ncu."""
    import torch
    import paper_2605_23571_gb300 as P
    P.build()
    # the FP32 product reads no FP64 stage states: leave the store out, so
    # that the device holds under a gigabyte for the profiler
    os.environ["EDA_STAGE_STORE"] = "0"
    dev = torch.device("cuda", 0)
    spec = replace(S.spec_scale(seed=0), n_members=args.profile_members, ckpt_every=args.profile_ckpt)
    spec = replace(spec, ell=min(spec.ell, spec.n_members - 1), k=min(spec.k, spec.n_members - 2))
    taps = P.bhalf_gaussian(spec.n, spec.length_scale, spec.sigma_b)
    dr = S.draws(spec)
    M, n, p = spec.n_members, spec.n, spec.p
    xb = torch.empty(M, n, dtype=torch.float64, device=dev)
    y = torch.empty(M, p, dtype=torch.float64, device=dev)
    with P.Handle.from_spec(replace(spec, ckpt_every=0), taps, precision=P.EDA_FP64) as hg:
        hg.eda_twin(torch.tensor(spec.F + spec.spin_sigma * dr.eta_spin, device=dev), spec.spinup,
                    torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
    cols = torch.arange(M, dtype=torch.int32, device=dev)
    V = torch.tensor(S.gaussian_matrix(M, n, 31), device=dev)
    hv = torch.empty_like(V)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED) as h:
        h.eda_set_trajectory(xb, y)
        h.eda_autotune(2)
        ms = h.eda_time_hvp_sweep(reps=3)
        h.eda_hvp(cols, V, hv, True)  # warm
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.eda_time_hvp_sweep(reps=1)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        plan = h.eda_sweep_plan(fp64=False)
    print(json.dumps({"profile_case": "scale", "workload": "l96_n65536_w96_m%d" % M, "members": M,
                      "ckpt_every": spec.ckpt_every, "ms_product": ms, "ms_profiled": e0.elapsed_time(e1),
                      "plan": plan, "algorithmic_bytes_full_trajectory": M * 4 * n * (2 * spec.nsteps + 2)}))
    return 0


def run_profile_lmp(args):
    """The LMP apply Z = R + S diag(c) S^T R of every member (Section 3.1) on
    CUDA cores (FP32 arithmetic, the mixed form's) and as split-BF16
    tensor-core products, timed with CUDA events at the scale size (n=65536,
    k=79, 81 members) and the batched size (n=4096, k=49, 51 members), on an
    orthonormal S with a decreasing spectrum loaded by eda_set_lmp (the apply
    does not read the trajectory, so the handles carry a 2-step window);
    then one tensor-core apply of each size inside a profiler range."""
    import torch
    import paper_2605_23571_gb300 as P
    P.build()
    os.environ["EDA_STAGE_STORE"] = "0"
    dev = torch.device("cuda", 0)
    out = {"profile_case": "lmp"}
    cases = (("scale", S.spec_small(65536, 2, 81, ell=80, k=79, length_scale=8.0, seed=5)),
             ("batched", S.spec_small(4096, 2, 51, ell=50, k=49, length_scale=8.0, seed=6)))
    hs = []
    for key, spec in cases:
        n, k, M = spec.n, spec.k, spec.n_members
        taps = P.bhalf_gaussian(n, spec.length_scale, spec.sigma_b)
        Sk = np.linalg.qr(S.gaussian_matrix(n, k, 7))[0]
        ev = np.logspace(5, 1, k)
        R = torch.tensor(S.gaussian_matrix(M, n, 8), device=dev)
        Z = torch.empty_like(R)
        h = P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED)
        h.eda_set_lmp(np.ascontiguousarray(Sk.T), ev)
        # algorithmic bytes of one apply: R read by both launches, Z written,
        # S read once in each of its two tiled BF16 forms (high and low parts)
        nS, kt = -(-n // 128) * 128, -(-k // 16) * 16
        res = {"n": n, "k": k, "members": M, "flops_per_apply": 4 * n * k * M,
               "bytes_per_apply_tc": 3 * 8 * n * M + 2 * 2 * nS * (128 + kt)}
        for kind, name in ((0, "cuda_cores_fp32"), (1, "tensor_cores_split_bf16")):
            for _ in range(3):
                h.eda_lmp_apply(R, Z, 0, kind)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                h.eda_lmp_apply(R, Z, 0, kind)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 20
            res[name] = {"ms": ms, "tflops": 4 * n * k * M / (ms / 1e3) / 1e12}
        res["tensor_cores_split_bf16"]["gbs"] = res["bytes_per_apply_tc"] / (res["tensor_cores_split_bf16"]["ms"] / 1e3) / 1e9
        out[key] = res
        hs.append((h, R, Z))
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for h, R, Z in hs:
        h.eda_lmp_apply(R, Z, 0, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    for h, _, _ in hs:
        h.close()
    print(json.dumps(out))
    return 0


def run_profile_hvp32(args):
    """The batched FP32 member Hessian product of the mixed form outside the
    persistent PCG: eda_hvp of all members (column j on member j's
    trajectory) on the autotuned tiling, twice untimed, then three times
    inside the profiler range, timed by CUDA events."""
    import torch
    import paper_2605_23571_gb300 as P
    P.build()
    dev = torch.device("cuda", 0)
    spec, dr = workload(args.seed)
    G = golden(spec, args.seed)
    taps = P.bhalf_gaussian(spec.n, spec.length_scale, spec.sigma_b)
    M, n, p = spec.n_members, spec.n, spec.p
    with P.Handle.from_spec(spec, taps, precision=P.EDA_MIXED) as h:
        xb = torch.empty(M, n, dtype=torch.float64, device=dev)
        y = torch.empty(M, p, dtype=torch.float64, device=dev)
        x0 = G["xt0"] if G is not None else spec.F + spec.spin_sigma * dr.eta_spin
        h.eda_twin(torch.tensor(x0, device=dev), 0 if G is not None else spec.spinup,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        rhs = torch.empty(M, n, dtype=torch.float64, device=dev)
        h.eda_set_trajectory(xb, y, rhs)
        h.eda_autotune(0)
        cols = torch.arange(M, dtype=torch.int32, device=dev)
        out = torch.empty_like(rhs)
        for _ in range(2):
            h.eda_hvp(cols, rhs, out, True)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            h.eda_hvp(cols, rhs, out, True)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        plan = h.eda_sweep_plan(fp64=False)
    print(json.dumps({"profile_case": "hvp32", "workload": spec.name, "members": M,
                      "ms_per_product": e0.elapsed_time(e1) / 3, "plan": plan}))
    return 0


def run_profile_case(args):
    """One fixed-iteration solve of the batched workload inside a profiler
    range: a small case of the solve's kernels for ncu (the same kernels and
    shapes as the timed steps, a few tens of milliseconds)."""
    if args.profile_case == "scale":
        return run_profile_scale(args)
    if args.profile_case == "lmp":
        return run_profile_lmp(args)
    if args.profile_case == "hvp32":
        return run_profile_hvp32(args)
    # one launch on the main tiling: no relaunch on the convergence tail's
    # tilings, whose members stop together after the fixed iterations
    os.environ["EDA_TAIL"] = "0"
    import torch
    import paper_2605_23571_gb300 as P
    P.build()
    dev = torch.device("cuda", 0)
    spec, dr = workload(args.seed)
    G = golden(spec, args.seed)
    taps = P.bhalf_gaussian(spec.n, spec.length_scale, spec.sigma_b)
    M, n, p = spec.n_members, spec.n, spec.p
    prec = P.EDA_FP64 if args.profile_case == "fp64" else P.EDA_MIXED
    with P.Handle.from_spec(spec, taps, precision=prec) as h:
        xb = torch.empty(M, n, dtype=torch.float64, device=dev)
        y = torch.empty(M, p, dtype=torch.float64, device=dev)
        x0 = G["xt0"] if G is not None else spec.F + spec.spin_sigma * dr.eta_spin
        h.eda_twin(torch.tensor(x0, device=dev), 0 if G is not None else spec.spinup,
                   torch.tensor(dr.eta_b, device=dev), torch.tensor(dr.eta_o, device=dev), xb, y)
        h.eda_set_trajectory(xb, y)
        h.eda_autotune(0)
        h.eda_sketch()
        h.eda_build_lmp()
        dz = torch.empty(M, n, dtype=torch.float64, device=dev)
        h.eda_solve_batch(0.0, args.profile_iters, None, True, dz)  # warm
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.eda_solve_batch(0.0, args.profile_iters, None, True, dz)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        plan = h.eda_sweep_plan(fp64=args.profile_case == "fp64")
    print(json.dumps({"profile_case": args.profile_case, "workload": spec.name, "iters": args.profile_iters,
                      "ms": e0.elapsed_time(e1), "plan": plan}))
    return 0


def main():
    args = parse()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
