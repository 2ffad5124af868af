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
    """The roofline of the dominant kernel: its launch time is the timed step time times its
    share of the profiled device time, its work the flop model; the cluster kernel's entry also
    carries the fraction of the peak of the SMs it occupies."""
    sys.path.insert(0, ROOT)
    import bench

    class W:
        name, batch, nx, ns = "single_64x128_imex", 1, 64, [128]

    prof = {"cluster_f64": (2.0, 20), "prep": (0.02, 1)}   # ms, launches in the profiled pass
    roof = bench.roofline_entry(prof, 0.05, W, 64, [128])
    share = 2.0 / 2.02
    assert roof["kernel"] == "cluster_f64" and abs(roof["share"] - share) < 1e-12
    ms = 0.05 * share / (20 / bench.PROFILE_STEPS)
    assert abs(roof["ms_per_launch"] - ms) < 1e-12
    fl = bench.kernel_flops("cluster_f64", 64, [128])
    assert abs(roof["achieved"] - fl / (ms / 1e3) / 1e12) < 1e-12
    assert roof["peak"] == bench.PEAK_TFLOPS["f64"] and roof["bound"] == "alu"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-15
    # the flop model of one tau-step: five 2-D transforms plus the pointwise terms
    assert fl == bench.step_flops(64, [128]) and 1.0e6 < fl < 1.3e6

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
