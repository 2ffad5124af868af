"""The benchmark's reference arm (the CPU oracle as the reference implementation) runs without a
GPU and prints one JSON line with the keys the bench contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.strip().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "single_64x128_imex"


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_roofline_entry_arithmetic():
    """The roofline of the dominant kernel: its launch time is the timed time per tau-step times
    its share of the profiled device time over its launches per tau-step; its work is the hot
    path's count (five unpruned real 2-D transforms of Nx Ns points at 2.5 N log2 N, plus 40
    flops per gridpoint) times the tau-steps per launch; the pruned count rides along."""
    sys.path.insert(0, ROOT)
    import bench

    class W:
        name, batch, nx, ns = "single_64x128_imex", 1, 64, [128]

    # profiled pass: 2000 tau-steps in 2 launches of the cluster kernel, plus a small kernel
    prof = {"cluster_f64": (72.0, 2), "prep": (0.02, 1)}   # ms, launches
    roof = bench.roofline_entry(prof, 2000, 0.036, W, 64, [128])
    share = 72.0 / 72.02
    assert roof["kernel"] == "cluster_f64" and abs(roof["share"] - share) < 1e-12
    assert roof["steps_per_launch"] == 1000
    ms = 0.036 * share / (2 / 2000)
    assert abs(roof["ms_per_launch"] - ms) < 1e-12
    fl = 1000 * (5 * 2.5 * 8192 * 13 + 40 * 8192)
    assert roof["flops_per_launch"] == fl == bench.survey_kernel_flops("cluster_f64", 64, [128], 1000)
    assert abs(roof["achieved"] - fl / (ms / 1e3) / 1e12) < 1e-12
    assert roof["peak"] == bench.PEAK_TFLOPS["f64"] and roof["bound"] == "alu"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-15
    # the pruned count of one tau-step: the complex transforms actually run plus pointwise terms
    fp = bench.kernel_flops("cluster_f64", 64, [128], 1000)
    assert fp == roof["flops_per_launch_pruned"] and 1.0e9 < fp < 1.3e9
    assert abs(roof["frac_pruned"] / roof["frac"] - fp / fl) < 1e-12
    # a per-phase kernel takes its phase's share of the step's count
    assert abs(sum(bench.survey_kernel_flops(k, 64, [128]) for k in
                   ("rows_nonlin", "cols_resid", "rows_adj", "cols_update"))
               - bench.survey_step_flops(64, [128])) < 1e-6

    class FakeK:
        KS_FP32 = 1

        @staticmethod
        def ks_get_option(handle, key):
            return {"path": 0, "cluster_f64": 16}[key]

    class H:
        handle = None

    class Props:
        multi_processor_count = 152

    import torch
    orig = torch.cuda.get_device_properties
    torch.cuda.get_device_properties = lambda dev: Props()
    try:
        r2 = bench.annotate_sms(dict(roof), FakeK, H, 0, 1, None)
    finally:
        torch.cuda.get_device_properties = orig
    assert r2["sms_used"] == 16 and abs(r2["frac_of_sms_used"] - roof["frac"] * 152 / 16) < 1e-15


def test_kernel_hash_ignores_comments_and_layout():
    """The traffic entries stay valid across comment and layout edits of the device code, and
    not across code edits."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) {\n    return x + 1;  // one more\n}\n/* note */"
    b = "int f(int x) { return x + 1; }  // reworded comment"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b) != bench.code_tokens(c)


def test_both_arms_name_the_same_config():
    """The two arms' lines carry identical config objects for the same workload."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2007_06427_gb300.inputs import workload
    w = workload("single_64x128_imex")
    c = bench.workload_config(w)
    assert set(c) == {"workload", "L", "nx", "ns", "batch", "gridpoints", "scheme", "dtau"}
    assert c["workload"] == "single_64x128_imex" and c["gridpoints"] == 8192


def test_rank_workloads_shard_one_recipe():
    """Under torchrun every rank gets a balanced shard of the workload's batch replicated per
    rank with the workload's own recipe (same Ns set, same T0 range); the shards are disjoint."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2007_06427_gb300.inputs import workload
    full = workload("ragged256_64xNs", seeds=range(2 * 8))
    parts = [bench.rank_workload("ragged256_64xNs", 8, 2, r) for r in range(2)]
    seen = set()
    for p in parts:
        for u, T, n in zip(p.u, p.T0, p.ns):
            assert n in (32, 64, 128, 256) and 10.0 <= T <= 100.0
            key = (n, round(T, 12))
            assert key not in seen
            seen.add(key)
    assert sum(p.batch for p in parts) == full.batch
    loads = [sum(p.ns) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(full.ns)
    one = bench.rank_workload("single_64x128_imex", None, 2, 1)
    assert one.batch == 1 and one.ns == [128] and one.T0[0] == workload("single_64x128_imex", seeds=[1]).T0[0]


def test_summary_is_compact_and_complete():
    sys.path.insert(0, ROOT)
    import bench
    tt = {"w": {"fp64": {"seconds": 1.23456, "total_steps": 10, "outcomes": {"converged": 1, "step_cap": 1}},
                "mixed": {"seconds": 0.5, "total_steps": 12, "outcomes": {"converged": 2}},
                "converged_in_every_variant": 1},
          "clocks": {"sm_mhz": 2070}}
    s = bench.summarize(tt)
    assert s == {"w": {"fp64": [1.235, 10, "1/2"], "mixed": [0.5, 12, "2/2"], "common": 1}}
