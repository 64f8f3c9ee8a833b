"""Host logic of bench.py (no GPU): the sweep-source hash that keys the ncu
traffic figure, the traffic lookup, and the kernel names of the tilings."""
import os

import bench

PLAN = dict(kind="cluster", ctas_per_vector=5, threads=256, C=4, K=8)


def test_code_hash_ignores_comments_and_blank_lines(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) {\n  return x + 1;\n}\n")
    b.write_text("// header\n/* block\n   comment */\nint f(int x) {  // trailing\n\n  return x + 1;\n}\n")
    c.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.code_sha256(str(a)) == bench.code_sha256(str(b))
    assert bench.code_sha256(str(a)) != bench.code_sha256(str(c))


def _profile(tmp_path, sha, plan="kind=cluster ctas_per_vector=5 threads=256 C=4 K=8"):
    p = tmp_path / "prof.md"
    p.write_text("captured plan: %s\nsweep.cu code sha256: %s\n"
                 "| dram bytes per launch (read + write): 1234567 | |\n" % (plan, sha))
    return str(p)


def test_traffic_only_for_the_captured_code_and_tiling(tmp_path, monkeypatch):
    src = tmp_path / "sweep.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "SWEEP_SRC", str(src))
    sha = bench.code_sha256(str(src))
    monkeypatch.setattr(bench, "SWEEP_PROFILE", _profile(tmp_path, sha))
    assert bench.sweep_traffic_per_launch(PLAN) == 1234567.0
    assert bench.sweep_traffic_per_launch(dict(PLAN, C=8)) is None      # another tiling
    assert bench.sweep_traffic_per_launch(dict(PLAN, kind="warp")) is None
    src.write_text("__global__ void k() { int x = 1; }\n")               # the code changed
    assert bench.sweep_traffic_per_launch(PLAN) is None
    monkeypatch.setattr(bench, "SWEEP_PROFILE", str(tmp_path / "missing.md"))
    assert bench.sweep_traffic_per_launch(PLAN) is None


def test_committed_profile_is_well_formed():
    # the committed summary names a tiling and a hash the lookup can parse
    assert os.path.exists(bench.SWEEP_PROFILE)
    txt = open(bench.SWEEP_PROFILE).read()
    assert "captured plan: kind=" in txt and "sweep.cu code sha256: " in txt
    assert "dram bytes per launch (read + write): " in txt


def test_kernel_names_follow_the_tiling():
    assert bench.sweep_kernel_name(PLAN).startswith("sweep_kernel<float,4> (clusters of 5 CTAs x 256 threads")
    assert bench.sweep_kernel_name(dict(PLAN, kind="warp", C=8)).startswith("wsweep_kernel<float,8>")
    assert "multi-launch" in bench.sweep_kernel_name(dict(PLAN, kind="multi-launch"), "double")


def test_cpu_baseline_all_cores_sample():
    # the oracle's PCG sample on several members at once in spawned workers
    import numpy as np

    import eda_synth as S
    import oracle as O
    spec = S.spec_small(200, 8, 5, every_var=2, every_step=2, length_scale=3.0, seed=3)
    taps = O.bhalf_taps(spec.n, spec.length_scale, spec.sigma_b)
    _, xb, y = O.twin(spec, S.draws(spec), taps)
    r = bench.cpu_oracle_step(spec, xb, y, taps, np.full(spec.n_members, 50), sample_iters=4, cores=2)
    ac = r["all_cores"]
    assert ac["cores"] == 2 and ac["t_full_step_s"] > r["t_setup_sketch_lmp_s"]
    # two members at once take less than twice one member's time per iteration
    t_seq = r["t_full_step_s"] - r["t_setup_sketch_lmp_s"]
    t_par = ac["t_full_step_s"] - r["t_setup_sketch_lmp_s"]
    assert t_par < 1.5 * t_seq


def test_profile_commands_run_on_this_bench():
    # every ncu summary under profiles/ names the bench.py command it was
    # taken with; each must still parse with this bench's options
    import glob
    import shlex
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    found = 0
    for path in glob.glob(os.path.join(root, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            if "python bench.py" not in line:
                continue
            args = shlex.split(line.split("python bench.py", 1)[1])
            bench.parse(args)  # raises SystemExit on an unknown option
            found += 1
    assert found >= 6
