#!/usr/bin/env python
"""Benchmark of the KS loop tau-descent on GB300: tau-step gridpoints/s and (unless --no-to-tol)
wall time to sqrt(J) < 1e-10, plain FP64 against FP32 bulk + FP64 finish.

One bench step is one tau-step of the whole hot path (residual, reductions, adjoint, update)
over the workload's batch, on the resident state in HBM.  The K timed steps run as the descent
driver runs them: ks_step launches of up to ``--chunk`` tau-steps each (the loop state stays in
shared memory inside a launch), each launch preceded by an L2 flush (a 256 MiB write) and timed
with CUDA events on the launch stream.  A latency line times one tau-step per launch the same
way.  Under torchrun the workload's batch is replicated per rank with the same recipe (seeds
continue across ranks) and sharded with shard.partition: every rank descends its own loops
(weak scaling, no collective on the data path); the reported time is the max over ranks.

Time to sqrt(J) < tol is measured on the single 64 x 128 loop, on a recurrence loop at the
paper's setting (L = 39, centre-symmetric) that converges to a periodic orbit, on the ragged
batch of 256 loops and on the 8 loops of 256 x 1024; a compact ``time_to_tol_summary`` closes
the JSON line.

``--impl reference`` times the CPU oracle (NumPy FP64, naive DFTs) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("τ-step gridpoints/s and time to ‖r‖<1e-10, mixed vs plain FP64, "
          "on 1 GB300")
UNIT = "gridpoint*tau-steps/s"
DEFAULT_WORKLOAD = "single_64x128_imex"

# Peaks: FP64 nominal from the GB300 table; FP32 from unit counts (152 SMs x 128 FP32 lanes x
# 2 flop/FMA) at the 2070 MHz maximum SM clock.
PEAK_TFLOPS = {"f64": 1.25, "f32": 152 * 128 * 2 * 2.070e9 / 1e12}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--chunk", type=int, default=1000,
                    help="tau-steps per timed launch (the descent driver's chunk)")
    ap.add_argument("--latency-steps", type=int, default=100,
                    help="one-step launches timed for the latency line (0: none)")
    ap.add_argument("--autotune", action="store_true",
                    help="create the timed handles with the autotuner (launch shape by timing)")
    ap.add_argument("--batch", type=int, default=None,
                    help="number of loops, for the batched workloads (default: the workload's)")
    ap.add_argument("--mode", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--e2e-tau-steps", type=int, default=100)
    ap.add_argument("--e2e-calls", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-to-tol", action="store_true",
                    help="skip every time-to-tolerance run")
    ap.add_argument("--no-fp32", action="store_true", help="skip the float-path throughput line")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the ragged-batch throughput line")
    ap.add_argument("--to-tol-max-steps", type=int, default=1_000_000)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--switch-tol", type=float, default=0.0,
                    help="mixed: switch to double once sqrt(J) (evaluated in double) <= this; "
                         "0: switch when it stops falling over the stall window")
    ap.add_argument("--orbit-max-steps", type=int, default=2_000_000,
                    help="step cap of the periodic-orbit descents (0: skip them)")
    ap.add_argument("--batched-max-steps", type=int, default=50_000,
                    help="step cap of the ragged-batch descents to tolerance (0: skip them)")
    ap.add_argument("--large-max-steps", type=int, default=20_000,
                    help="step cap of the 256 x 1024 descents to tolerance (0: skip them)")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="K",
                    help="profiling case: load the workload, run 3 x K tau-steps, no timing")
    ap.add_argument("--ncu-dns", type=int, default=0, metavar="K",
                    help="profiling case: K steps of the batched KSE run (1216 trajectories, "
                         "L = 39, 64 modes), no timing")
    ap.add_argument("--no-dns", action="store_true", help="skip the chaotic-run (DNS) line")
    ap.add_argument("--path", type=int, default=-1,
                    help="profiling case: launch path (0 cluster, 1 persistent, 2 per-phase)")
    ap.add_argument("--no-graph", action="store_true",
                    help="profiling case: launch the per-phase kernels directly, not as CUDA graphs")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------------
# algorithmic work per launch
# ---------------------------------------------------------------------------------------
def dns_step_flops(nx: int) -> float:
    """Algorithmic flops of one ETDRK4 step of one trajectory of the KSE run: four nonlinear
    evaluations, each an inverse and a forward complex transform of Nx points shared by two
    trajectories (5 N log2 N flops each, so 20 Nx log2 Nx per trajectory), the square on the grid
    (Nx), the split and the -(i q / 2) factor (6 per retained mode), and the scheme's stage
    combinations (52 per retained mode)."""
    nh = nx // 3 + 1
    return 20.0 * nx * math.log2(nx) + 4.0 * (nx + 6.0 * nh) + 52.0 * nh


def survey_step_flops(nx: int, nss) -> float:
    """Algorithmic flops of one tau-step of the batch by the hot path's work count: five 2-D real
    transforms of Nx Ns points, each 2.5 N log2 N flops (an unpruned real FFT), plus 40 flops per
    gridpoint for the spectral and pointwise terms."""
    return sum(5 * 2.5 * nx * n * math.log2(nx * n) + 40.0 * nx * n for n in nss)


def fft_flops(n: int) -> float:
    return 5.0 * n * math.log2(n)


def kernel_flops(kind: str, nx: int, nss, steps_per_launch: int = 1) -> float:
    """Flops of one launch of `kind` by the pruned count: every complex transform the kernels
    actually run (5 n log2 n), only over the retained x-modes in s, plus the pointwise terms.

    Fused kernels (cluster-resident, grid-persistent) run whole tau-steps: their work is the
    sum of the four phases times the steps per launch."""
    if kind.startswith("cluster") or kind.startswith("persist"):
        return steps_per_launch * step_flops(nx, nss)
    nkx = nx // 3 + 1
    rows = sum(nss)
    if kind.startswith("rows_nonlin"):
        # one inverse transform of u + i u_x per row, product, one forward per row pair
        return rows * (1.5 * fft_flops(nx) + 2.0 * nx)
    if kind.startswith("rows_adj"):
        # one inverse (r_x pair) and one forward (u r_x pair) per row pair, product
        return rows * (1.0 * fft_flops(nx) + 2.0 * nx)
    if kind.startswith("cols_resid"):
        return sum(nkx * (2 * fft_flops(n) + 24.0 * (2 * (n // 3) + 1)) for n in nss)
    if kind.startswith("cols_update"):
        return sum(nkx * (2 * fft_flops(n) + 30.0 * (2 * (n // 3) + 1)) for n in nss)
    return 0.0


def survey_kernel_flops(kind: str, nx: int, nss, steps_per_launch: int = 1) -> float:
    """Flops of one launch by the hot path's work count (``survey_step_flops``); a per-phase
    kernel takes the share of the step that the pruned count gives its phase."""
    if kind.startswith("cluster") or kind.startswith("persist"):
        return steps_per_launch * survey_step_flops(nx, nss)
    pruned = step_flops(nx, nss)
    return kernel_flops(kind, nx, nss) * survey_step_flops(nx, nss) / pruned if pruned else 0.0


def code_tokens(src: str) -> str:
    """C++ source without its comments and with whitespace collapsed: what the compiler sees
    (the device sources hold no string literal with a comment marker in it)."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash() -> str:
    """Hash of the device code of the fused kernels (the per-CTA items and the cluster-resident
    kernel), comments and layout excluded; host-side changes leave it unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in ("ks_items.cuh", "ks_cluster.cuh"):
        with open(os.path.join(ROOT, "paper_2007_06427_gb300", "csrc", f)) as fh:
            h.update(code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, kernel: str, steps_per_launch: int = 1):
    """DRAM bytes per launch from the committed ncu capture, if the CUDA sources still match and
    the capture ran the same number of tau-steps per launch."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_sha") != kernel_source_hash():
        return None
    e = t.get("kernels", {}).get(f"{workload}/{kernel}/{steps_per_launch}")
    return None if e is None else e.get("bytes_per_launch")


def step_flops(nx, nss) -> float:
    return sum(kernel_flops(k, nx, nss) for k in ("rows_nonlin", "cols_resid", "rows_adj",
                                                   "cols_update"))


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# CPU oracle timing (runs in a fresh interpreter: single-threaded BLAS, no CUDA context)
# ---------------------------------------------------------------------------------------
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import ks_oracle as ko
from paper_2007_06427_gb300.inputs import workload
w = workload({wl!r}, {batch!r})
gs = [ko.grid(w.nx, n, w.L) for n in w.ns]
uh = [ko.band_state(u, w.L) for u in w.u]
T = list(w.T0)
for b in range(w.batch):                      # warm-up step (builds DFT matrices)
    ko.step_hat(uh[b], T[b], gs[b], w.dtau, w.scheme)
mode = {mode!r}
t0 = time.perf_counter()
steps = 0
gp = 0
budget = {budget!r}
max_steps = {max_steps!r}
while True:
    for b in range(w.batch):
        uh[b], T[b], _, _ = ko.step_hat(uh[b], T[b], gs[b], w.dtau, w.scheme)
        gp += w.ns[b] * w.nx
    steps += 1
    el = time.perf_counter() - t0
    if (budget and el >= budget) or (max_steps and steps >= max_steps):
        break
print(json.dumps({{"steps": steps, "seconds": el, "gridpoint_steps": gp}}))
"""


def run_cpu_oracle(workload_name: str, budget_s: float = 0.0, max_steps: int = 0,
                   threads: int = 1, batch=None):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = CPU_SNIPPET.format(root=ROOT, wl=workload_name, batch=batch, mode="fp64", budget=budget_s,
                              max_steps=max_steps)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def workload_config(w) -> dict:
    """The workload as both arms name it (identical keys and values in both lines)."""
    return {"workload": w.name, "L": w.L, "nx": w.nx, "ns": w.ns[:8], "batch": w.batch,
            "gridpoints": w.gridpoints, "scheme": "imex" if w.scheme else "explicit",
            "dtau": w.dtau}


def rank_workload(name: str, batch, ws: int, rank: int):
    """This rank's loops: the workload's batch replicated ws times with the same recipe (seeds
    0 .. ws * B - 1) and sharded with shard.partition (longest loops first, balanced by
    Ns * Nx); weak scaling, every rank about one workload's batch."""
    from paper_2007_06427_gb300.inputs import workload
    from paper_2007_06427_gb300 import shard
    base = workload(name, batch)
    if ws == 1:
        return base
    full = workload(name, seeds=range(ws * base.batch))
    mine = shard.partition(full.ns, full.nx, ws)[rank]
    return workload(name, seeds=mine)


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2007_06427_gb300.inputs import workload
    w = workload(args.workload, args.batch)
    # warm-up steps, then exactly K timed oracle tau-steps
    if args.warmup:
        run_cpu_oracle(args.workload, 0.0, args.warmup, batch=args.batch)
    r = run_cpu_oracle(args.workload, 0.0, args.steps, batch=args.batch)
    value = r["gridpoint_steps"] / r["seconds"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * r["seconds"] / r["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{r['steps']} oracle tau-steps of the workload (NumPy FP64 "
                                   "dense DFTs, single-threaded BLAS)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_launches(K, h, nsteps: int, chunk: int, flush, stream, no_flush: bool):
    """nsteps tau-steps of the resident state in launches of up to `chunk` steps, each after an
    L2 flush, each timed with CUDA events on the launch stream.  Returns [(ms, steps)]."""
    import torch
    evs = []
    done = 0
    while done < nsteps:
        c = min(chunk, nsteps - done)
        if not no_flush:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.ks_step(h.handle, c, 0.0, stream)
        e1.record(stream)
        evs.append((e0, e1, c))
        done += c
    torch.cuda.synchronize()
    return [(a.elapsed_time(b), c) for a, b, c in evs]


def profile_pass(K, h, nsteps: int, chunk: int, flush, stream, no_flush: bool):
    """An untimed pass with the same launch pattern and the library's per-kernel event timing
    on.  Returns ({kind: (ms, launches)}, library launches, tau-steps).  The timed region runs
    without the library's own events, which would add device work to every launch."""
    K.ks_profile(h.handle, True)
    K.ks_profile_read(h.handle, reset=True)
    timed_launches(K, h, nsteps, chunk, flush, stream, no_flush)
    prof, launches = K.ks_profile_read(h.handle, reset=True)
    K.ks_profile(h.handle, False)
    return prof, launches, nsteps


def roofline_entry(prof, prof_steps: int, ms_per_step: float, w, nx, nss):
    """Roofline of the dominant kernel.  Its mean launch duration is the timed region's time per
    tau-step (CUDA events on the launch stream) times its share of the library's device time in
    the profiled pass, divided by its launches per tau-step; its work is the hot path's flop
    count (five unpruned real 2-D transforms plus 40 flops per gridpoint per tau-step), the
    pruned count of the transforms actually run given beside it."""
    dname = max(prof, key=lambda k: prof[k][0]) if prof else None
    if not dname:
        return None
    ms_k, cnt = prof[dname]
    tot = max(sum(v[0] for v in prof.values()), 1e-30)
    share = ms_k / tot
    launches_per_step = cnt / prof_steps
    steps_per_launch = 1.0 / launches_per_step if dname[:7] in ("cluster", "persist") else 1
    ms_launch = ms_per_step * share / max(launches_per_step, 1e-30)
    spl = int(round(steps_per_launch))
    fl = survey_kernel_flops(dname, nx, nss, spl)
    fl_pruned = kernel_flops(dname, nx, nss, spl)
    ach = fl / (ms_launch / 1e3) / 1e12 if ms_launch > 0 else 0.0
    pk = PEAK_TFLOPS["f32" if "_f32" in dname and "adj" not in dname else "f64"]
    trf = measured_traffic(w.name, dname, spl)
    return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
            "frac": ach / pk, "traffic": trf, "kernel": dname,
            "flops_per_launch": fl, "steps_per_launch": spl, "ms_per_launch": ms_launch,
            "ms_per_launch_profiled": ms_k / cnt, "share": share,
            "flops_per_launch_pruned": fl_pruned,
            "frac_pruned": fl_pruned / (ms_launch / 1e3) / 1e12 / pk if ms_launch > 0 else 0.0,
            "peak_source": ("nominal GB300 FP64 rate (1.25 TFLOP/s)" if pk == PEAK_TFLOPS["f64"]
                            else "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz")}


def annotate_sms(roof, K, h, mode, batch, dev):
    """For the cluster-resident kernel: the SMs a launch occupies (one CTA per SM; C CTAs per
    loop) and the roofline fraction against the peak of those SMs alone."""
    import torch
    if not roof or K.ks_get_option(h.handle, "path") != 0:
        return roof
    C = K.ks_get_option(h.handle, "cluster_f32" if mode == K.KS_FP32 else "cluster_f64")
    if C <= 0:
        return roof
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    used = min(n_sms, C * batch)
    roof["sms_used"] = used
    roof["frac_of_sms_used"] = roof["frac"] * n_sms / used
    return roof


def add_probe(roof, probe):
    """The measured pipe peak of the roofline's precision (the library's FMA probe) and the
    fraction of it, beside the nominal ones."""
    if not roof:
        return
    key = "f64" if roof["peak"] == PEAK_TFLOPS["f64"] else "f32"
    p = probe.get(key)
    roof["peak_probe"] = p
    roof["frac_of_probe"] = roof["achieved"] / p if p else None


def launch_shape(K, h, mode, autotuned):
    sfx = "f32" if mode == K.KS_FP32 else "f64"
    path = K.ks_get_option(h.handle, "path")
    cl = path == 0 and K.ks_get_option(h.handle, "cluster_" + sfx) > 0  # the cluster kernel runs
    return {"path": path,
            "cluster": K.ks_get_option(h.handle, "cluster_" + sfx),
            "threads": K.ks_get_option(h.handle, "cluster_threads"),
            # the cluster kernel's block, exchange form and launch-bound variant
            "cluster_block": K.ks_get_option(h.handle, "cluster_block_" + sfx) if cl else None,
            "exchange": (("mbarrier" if K.ks_get_option(h.handle, "cluster_exchange_" + sfx)
                          else "cluster barrier") if cl else None),
            "min_blocks": K.ks_get_option(h.handle, "cluster_min_blocks_" + sfx) if cl else None,
            "graph": K.ks_get_option(h.handle, "graph"),
            "graph_replays": K.ks_get_option(h.handle, "graph_replays"),
            "autotuned": bool(autotuned)}


def throughput(args, w, mode, dev, flush, K, nsteps, autotune=False, latency_steps=0):
    """The steady-state line of one handle: nsteps tau-steps in launches of args.chunk, each
    after a flush; plus, if latency_steps, one-step launches (the latency of a single step)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.from_numpy(w.packed()).to(dev, dt)
    T = torch.tensor(w.T0, dtype=torch.float64, device=dev)
    h = K.KSLoop(w.L, w.nx, w.ns, mode, w.scheme, w.dtau, autotune=int(autotune))
    if w.meta.get("symmetry"):
        K.ks_set_option(h.handle, "symmetry", 1)
    K.ks_set_state(h.handle, u, T, stream)
    # warm-up: W tau-steps in the timed launch pattern (untimed)
    timed_launches(K, h, args.warmup, args.chunk, flush, stream, args.no_flush)
    prof, plaunch, psteps = profile_pass(K, h, min(nsteps, 2 * args.chunk), args.chunk, flush,
                                         stream, args.no_flush)
    out = {"h": h, "prof": prof, "prof_steps": psteps, "launches_per_step": plaunch / psteps}
    if latency_steps:
        lprof, ll, ls_ = profile_pass(K, h, latency_steps, 1, flush, stream, args.no_flush)
        lt = timed_launches(K, h, latency_steps, 1, flush, stream, args.no_flush)
        lms = sum(m for m, _ in lt) / latency_steps
        lroof = roofline_entry(lprof, ls_, lms, w, w.nx, w.ns)
        out["latency"] = {"value": w.gridpoints / (lms / 1e3), "unit": UNIT,
                          "ms_per_step": lms, "steps": latency_steps,
                          "note": "one tau-step per launch, L2 flushed before each",
                          "roofline": annotate_sms(lroof, K, h, mode, w.batch, dev)}
    out["events"] = timed_launches(K, h, nsteps, args.chunk, flush, stream, args.no_flush)
    return out


def ours_arm(args):
    import numpy as np
    import torch
    from paper_2007_06427_gb300 import ks_loop as K

    ws, rank, lrank = dist_env()
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    # CPU baseline before any GPU work (fresh interpreter, spawned)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            r = run_cpu_oracle(args.workload, args.cpu_seconds, 0, batch=args.batch)
            cpu = {"value": r["gridpoint_steps"] / r["seconds"], "unit": UNIT, "cores": 1,
                   "kind": "oracle",
                   "sample": f"{r['steps']} oracle tau-steps of {args.workload} "
                             f"({r['seconds']:.1f} s, NumPy FP64 dense DFTs, 1 BLAS thread)"}
            nc = os.cpu_count() or 1
            if nc > 1:
                ra = run_cpu_oracle(args.workload, args.cpu_seconds / 2, 0, threads=nc,
                                    batch=args.batch)
                cpu["all_cores"] = {"value": ra["gridpoint_steps"] / ra["seconds"], "cores": nc,
                                    "sample": f"{ra['steps']} oracle tau-steps, {nc} BLAS threads"}
        except Exception as e:  # keep the GPU line even if the host leg fails
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"failed: {str(e)[-200:]}"}

    # the FP64 and FP32 pipe peaks of this GPU, measured by the library's FMA probe (context for
    # the roofline fractions, which are taken against the nominal rates)
    probe = {}
    for key, prec in (("f64", K.KS_FP64), ("f32", K.KS_FP32)):
        try:
            probe[key] = K.ks_probe_peak(prec)
        except Exception:  # keep the line if the probe fails
            probe[key] = None
    w = rank_workload(args.workload, args.batch, ws, rank)
    mode = K.KS_FP32 if args.mode == "fp32" else K.KS_FP64
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    nx, nss = w.nx, w.ns
    gp = w.gridpoints
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(lrank)
    clk.start()
    tp = throughput(args, w, mode, dev, flush, K, args.steps, args.autotune,
                    args.latency_steps if ws == 1 else 0)
    clocks = clk.stop()
    if pg:
        pg.barrier()
    h = tp["h"]
    total_ms = sum(m for m, _ in tp["events"])
    launches = int(round(tp["launches_per_step"] * args.steps))
    tmax = total_ms
    if pg:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        tmax = float(t.item())
    if pg:
        g = torch.tensor([float(gp)], dtype=torch.float64, device=dev)
        pg.all_reduce(g)
        gp_all = float(g.item())
    else:
        gp_all = float(gp)
    value = gp_all * args.steps / (tmax / 1e3)
    roof = annotate_sms(roofline_entry(tp["prof"], tp["prof_steps"], total_ms / args.steps,
                                       w, nx, nss), K, h, mode, w.batch, dev)

    # end to end through the public call with pinned host buffers
    e2e = None
    if args.e2e_calls > 0:
        E = args.e2e_tau_steps
        hu = torch.from_numpy(w.packed()).to(dt).pin_memory()
        hT = torch.tensor(w.T0, dtype=torch.float64).pin_memory()
        hs = torch.zeros(w.batch, dtype=torch.int64).pin_memory()
        hq = torch.zeros(w.batch, dtype=torch.float64).pin_memory()
        hst = torch.zeros(w.batch, dtype=torch.int32).pin_memory()
        u0 = hu.clone()
        T0 = hT.clone()
        K.ks_descend(h.handle, hu.numpy(), hT.numpy(), E, 0.0, hs.numpy(), hq.numpy(), hst.numpy())
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_calls):
            hu.copy_(u0)
            hT.copy_(T0)
            K.ks_descend(h.handle, hu.numpy(), hT.numpy(), E, 0.0, hs.numpy(), hq.numpy(),
                         hst.numpy())
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        if pg:
            t = torch.tensor([el], dtype=torch.float64, device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            el = float(t.item())
        ub = hu.numel() * hu.element_size()
        e2e = {"value": gp_all * E * args.e2e_calls / el, "unit": UNIT,
               "h2d_bytes_per_step": ub + 8 * w.batch,
               "d2h_bytes_per_step": ub + (8 + 8 + 8 + 4) * w.batch,
               "tau_steps_per_call": E,
               "note": "one bench step = one ks_descend call on pinned host buffers"}
    shape = launch_shape(K, h, mode, args.autotune)
    h.close()

    fp32 = None
    if not args.no_fp32 and mode == K.KS_FP64 and ws == 1:
        t32 = throughput(args, w, K.KS_FP32, dev, flush, K, args.steps)
        ms32 = sum(m for m, _ in t32["events"])
        fp32 = {"value": gp * args.steps / (ms32 / 1e3), "unit": UNIT,
                "ms_per_step": ms32 / args.steps, "dtype": "f32",
                "gpu_launches": int(round(t32["launches_per_step"] * args.steps)),
                "roofline": annotate_sms(roofline_entry(t32["prof"], t32["prof_steps"],
                                                        ms32 / args.steps, w, nx, nss),
                                         K, t32["h"], K.KS_FP32, w.batch, dev)}
        t32["h"].close()

    batched = None
    if not args.no_batched and ws == 1 and args.workload != "ragged256_64xNs":
        batched = batched_line(args, dev, flush, K)

    dns = None
    if not args.no_dns and ws == 1:
        dns = dns_line(dev, flush, K)
        add_probe((dns.get("batch1216") or {}).get("roofline"), probe)

    to_tol = None
    if not args.no_to_tol and ws == 1:
        to_tol = run_to_tol(args, w, dev, K)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if mode == K.KS_FP32 else "f64", "data": "synthetic",
            "config": workload_config(w),
            "timing": {"l2": "flushed (256 MiB write) before every timed launch",
                       "tau_steps_per_launch": min(args.chunk, args.steps),
                       "launch": shape},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "kernels_profiled_pass": {k: {"ms": v[0], "launches": v[1]} for k, v in tp["prof"].items()},
        }
        for entry in (roof, (fp32 or {}).get("roofline"), (batched or {}).get("roofline"),
                      tp.get("latency", {}).get("roofline")):
            add_probe(entry, probe)
        if "latency" in tp:
            line["latency"] = tp["latency"]
        if fp32:
            line["fp32"] = fp32
        if batched:
            line["batched"] = batched
        if dns:
            line["dns"] = dns
        if to_tol:
            attach_cpu_extrapolation(to_tol, cpu, w)
            line["time_to_tol"] = to_tol
            line["time_to_tol_summary"] = summarize(to_tol)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def batched_line(args, dev, flush, K):
    """Throughput of the ragged batch of 256 loops (Nx = 64, Ns from {32, 64, 128, 256}) in
    FP64 on the launch shape the autotuner picks, with its own roofline entry."""
    from paper_2007_06427_gb300.inputs import workload
    w = workload("ragged256_64xNs")
    n = max(20, min(args.steps, 200))
    t = throughput(args, w, K.KS_FP64, dev, flush, K, n, autotune=True)
    ms = sum(m for m, _ in t["events"])
    # the whole step against the FP64 peak (the autotuner may pick four launches per step, whose
    # phases the hot path's work count does not split)
    fl = survey_step_flops(w.nx, w.ns)
    ach = fl / (ms / n / 1e3) / 1e12
    fl_p = step_flops(w.nx, w.ns)
    roof = {"bound": "alu", "achieved": ach, "peak": PEAK_TFLOPS["f64"], "unit": "TFLOP/s",
            "frac": ach / PEAK_TFLOPS["f64"], "traffic": None,
            "kernel": "every kernel of a tau-step", "flops_per_step": fl,
            "flops_per_step_pruned": fl_p,
            "frac_pruned": fl_p / (ms / n / 1e3) / 1e12 / PEAK_TFLOPS["f64"],
            "kernels": {k: v[0] / max(sum(x[0] for x in t["prof"].values()), 1e-30)
                        for k, v in t["prof"].items()},
            "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)"}
    out = {"workload": w.name, "value": w.gridpoints * n / (ms / 1e3), "unit": UNIT,
           "ms_per_step": ms / n, "steps": n, "dtype": "f64",
           "launch": launch_shape(K, t["h"], K.KS_FP64, True), "roofline": roof}
    t["h"].close()
    return out


def outcome_counts(K, st):
    """Loops of the batch per final status (converged, step cap, stalled, diverged)."""
    out = {}
    for v in st.tolist():
        name = K.STATUS_NAMES.get(int(v), str(int(v)))
        out[name] = out.get(name, 0) + 1
    return out


def descend_variant(K, w, dev, mode, tol, cap, *, switch_tol=0.0, extrapolate=False,
                    f32_adjoint=None, symmetry=False, chunk=None, u_override=None):
    """One descent of the whole batch from its initial loops to sqrt(J) < tol or the cap; returns
    a record with the wall time, per-loop outcomes and the classes reached."""
    import numpy as np
    import torch
    from paper_2007_06427_gb300.orbits import classify
    ck = chunk or (1000 if extrapolate else 2000)
    h = K.KSLoop(w.L, w.nx, w.ns, mode, w.scheme, w.dtau, tol=tol, switch_tol=switch_tol,
                 max_steps=cap, chunk=ck)
    if extrapolate:
        K.ks_set_option(h.handle, "extrapolate", 1)
    if symmetry:
        K.ks_set_option(h.handle, "symmetry", 1)
    if f32_adjoint is not None:
        K.ks_set_option(h.handle, "finish_f32_adjoint", int(f32_adjoint))
    packed = w.packed() if u_override is None else u_override
    u = torch.from_numpy(packed).to(dev, torch.float64)
    T = torch.tensor(w.T0, dtype=torch.float64, device=dev)
    steps = torch.zeros(w.batch, dtype=torch.int64, device=dev)
    sq = torch.zeros(w.batch, dtype=torch.float64, device=dev)
    st = torch.zeros(w.batch, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    K.ks_descend(h.handle, u, T, cap, tol, steps, sq, st)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    hs, hq, hp = K.ks_get_history(h.handle, 0)
    uo = u.cpu().numpy()
    kinds, off = {}, 0
    conv = []
    for b, n in enumerate(w.ns):
        kind, _, _ = classify(uo[off:off + n * w.nx].reshape(n, w.nx), w.L)
        off += n * w.nx
        if int(st[b]) == K.KS_CONVERGED:
            kinds[kind] = kinds.get(kind, 0) + 1
            conv.append(b)
    rec = {"seconds": el, "total_steps": int(steps.sum().item()),
           "outcomes": outcome_counts(K, st), "converged_classes": kinds,
           "converged_loops": conv if len(conv) <= 16 else len(conv),
           "steps": steps.tolist()[:8], "sqrtJ": sq.tolist()[:8], "T": T.tolist()[:8],
           "switch_tol": switch_tol, "extrapolate": bool(extrapolate), "cap": cap,
           "gridpoint_steps": int(sum(int(a) * n * w.nx for a, n in zip(steps.tolist(), w.ns)))}
    if mode == K.KS_MIXED:
        rec["finish_f32_adjoint"] = K.ks_get_option(h.handle, "finish_f32_adjoint")
        rec["loop0_switch_step"] = int(hs[np.nonzero(hp == 0)[0][0]]) if (hp == 0).any() else None
    if extrapolate:
        rec["extrapolations"] = K.ks_get_option(h.handle, "extrapolations")
        rec["rejected"] = K.ks_get_option(h.handle, "extrapolations_rejected")
    marks = {}
    for target in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10):
        idx = np.nonzero(hq < target)[0]
        if idx.size:
            marks[f"{target:.0e}"] = int(hs[idx[0]])
    rec["loop0_first_step_below"] = marks
    rec["_st"] = st.cpu().numpy()
    h.close()
    return rec


def run_to_tol(args, w, dev, K):
    """Plain FP64 descent against FP32 bulk + FP64 finish, from the same loops, to sqrt(J) < tol,
    with and without the extrapolation of App. C, on: the bench workload; a recurrence loop at
    the paper's setting that reaches a periodic orbit; the ragged batch of 256 loops; the eight
    256 x 1024 loops (FP32 to 1e-5, then FP64).  Batched runs stop at a stated step cap."""
    from paper_2007_06427_gb300.inputs import orbit_guess, workload
    out = {}
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    clk.start()
    cap, tol = args.to_tol_max_steps, args.tol
    single = {}
    single["fp64"] = descend_variant(K, w, dev, K.KS_FP64, tol, cap)
    single["mixed"] = descend_variant(K, w, dev, K.KS_MIXED, tol, cap, switch_tol=args.switch_tol)
    # the finishing steps with the descent direction formed in float (knob finish_f32_adjoint)
    single["mixed_f32_adjoint_finish"] = descend_variant(K, w, dev, K.KS_MIXED, tol, cap,
                                                         switch_tol=args.switch_tol, f32_adjoint=1)
    single["fp64_extrapolated"] = descend_variant(K, w, dev, K.KS_FP64, tol, cap, extrapolate=True)
    # the extrapolated mixed run switches to double at sqrt(J) = 1e-5, about the float floor of
    # this loop: the jumps of the extrapolation restart the stall window the plain run waits on
    single["mixed_extrapolated"] = descend_variant(K, w, dev, K.KS_MIXED, tol, cap,
                                                   switch_tol=max(args.switch_tol, 1e-5),
                                                   extrapolate=True)
    out[w.name] = single
    if args.orbit_max_steps > 0:
        g = orbit_guess()
        oc = args.orbit_max_steps
        orb = {"note": "centre-symmetric recurrence loop of a chaotic run at L = 39 (T0 = %.2f), "
                       "descended with the symmetry knob; the paper lists a periodic orbit of "
                       "period 25.37 at this setting (Sec. 4.4)" % g.T0[0]}
        for name, mode, ext in (("fp64", K.KS_FP64, False), ("mixed", K.KS_MIXED, False),
                                ("fp64_extrapolated", K.KS_FP64, True),
                                ("mixed_extrapolated", K.KS_MIXED, True)):
            orb[name] = descend_variant(K, g, dev, mode, tol, oc, extrapolate=ext, symmetry=True,
                                        switch_tol=1e-5 if (ext and mode == K.KS_MIXED) else 0.0)
        # the finishing steps with the descent direction formed in float
        orb["mixed_f32_adjoint_finish"] = descend_variant(K, g, dev, K.KS_MIXED, tol, oc,
                                                          symmetry=True, f32_adjoint=1)
        out[g.name] = orb
    if args.batched_max_steps > 0:
        rg = workload("ragged256_64xNs")
        bc = args.batched_max_steps
        bt = {}
        for name, mode, ext in (("fp64_extrapolated", K.KS_FP64, True),
                                ("mixed_extrapolated", K.KS_MIXED, True)):
            bt[name] = descend_variant(K, rg, dev, mode, tol, bc, extrapolate=ext,
                                       switch_tol=1e-5 if mode == K.KS_MIXED else 0.0)
        out[rg.name] = bt
    if args.large_max_steps > 0:
        lg = workload("large8_256x1024")
        lc = args.large_max_steps
        lt = {"fp64": descend_variant(K, lg, dev, K.KS_FP64, tol, lc),
              "fp32_then_fp64": descend_variant(K, lg, dev, K.KS_MIXED, tol, lc, switch_tol=1e-5)}
        out[lg.name] = lt
    for grp in out.values():
        common = None
        for k, v in grp.items():
            if isinstance(v, dict) and "_st" in v:
                conv = set(int(i) for i in (v["_st"] == K.KS_CONVERGED).nonzero()[0])
                common = conv if common is None else common & conv
        for k, v in list(grp.items()):
            if isinstance(v, dict) and "_st" in v:
                del v["_st"]
        if common is not None:
            grp["converged_in_every_variant"] = len(common)
    out["clocks"] = clk.stop()
    return out


def attach_cpu_extrapolation(to_tol, cpu, w):
    """The oracle at its measured per-step rate for the step counts of the FP64 descents of the
    bench workload (labelled as extrapolated), and each variant's achieved flop rate."""
    grp = to_tol.get(w.name, {})
    for key, v in grp.items():
        if not isinstance(v, dict) or "seconds" not in v:
            continue
        if cpu and cpu.get("value") and key.startswith("fp64"):
            v["cpu_oracle_seconds_extrapolated"] = v["gridpoint_steps"] / cpu["value"]
        if v["seconds"] > 0:
            ach = survey_step_flops(w.nx, w.ns) / w.gridpoints * v["gridpoint_steps"] / v["seconds"] / 1e12
            v["achieved_tflops"] = ach
            if key.startswith("fp64"):
                v["frac_of_fp64_peak"] = ach / PEAK_TFLOPS["f64"]


def summarize(to_tol) -> dict:
    """Compact record of every time-to-tolerance variant: [seconds, total tau-steps of the batch,
    loops converged / batch]."""
    out = {}
    for wl, grp in to_tol.items():
        if not isinstance(grp, dict) or wl == "clocks":
            continue
        row = {}
        for k, v in grp.items():
            if isinstance(v, dict) and "seconds" in v:
                n = sum(v["outcomes"].values())
                row[k] = [round(v["seconds"], 3), v["total_steps"],
                          f"{v['outcomes'].get('converged', 0)}/{n}"]
        if "converged_in_every_variant" in grp:
            row["common"] = grp["converged_in_every_variant"]
        out[wl] = row
    return out


def dns_line(dev, flush, K):
    """The chaotic run behind the initial loops (Sec. 4.3) on the GPU (ks_dns): the paper-length
    run (L = 39, 64 modes, dt = 0.25, t = 6000, one trajectory, saved every 2 steps) and a batch
    of 1216 trajectories (eight per block on every SM), each launch after an L2 flush and timed
    with CUDA events; gridpoint-steps/s and the FP64 roofline of the batched run."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    L, nx, dt = 39.0, 64, 0.25
    for name, B, nsteps in (("single_t6000", 1, 24000), ("batch1216", 1216, 4000)):
        rng = np.random.default_rng(7)
        u0 = torch.tensor(0.1 * rng.standard_normal((B, nx)), device=dev)
        nsave = nsteps // 2 + 1
        us = torch.empty(B, nsave, nx, dtype=torch.float64, device=dev)
        nrm = torch.empty(B, nsave, dtype=torch.float64, device=dev)
        K.ks_dns(L, nx, B, dt, 200, 2, True, u0, us, nrm, None, stream)   # warm-up
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        K.ks_dns(L, nx, B, dt, nsteps, 2, True, u0, us, nrm, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ent = {"trajectories": B, "steps": nsteps, "ms": ms, "us_per_step": 1e3 * ms / nsteps,
               "value": B * nx * nsteps / (ms / 1e3), "unit": "gridpoint*steps/s"}
        if B > 1:
            ach = B * nsteps * dns_step_flops(nx) / (ms / 1e3) / 1e12
            ent["roofline"] = {"bound": "alu", "achieved": ach, "peak": PEAK_TFLOPS["f64"],
                               "unit": "TFLOP/s", "frac": ach / PEAK_TFLOPS["f64"],
                               "traffic": None, "kernel": "k_dns",
                               "flops_per_launch": B * nsteps * dns_step_flops(nx),
                               "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)"}
        out[name] = ent
    out["note"] = ("ETDRK4 of the KSE, L = 39, 64 modes, dt = 0.25, centre-symmetric, state "
                   "saved every 2 steps with its norm; one launch per run")
    return out


def ncu_dns(args):
    """Small fixed case for ncu captures of the KSE run: 1216 trajectories, K steps."""
    import numpy as np
    import torch
    from paper_2007_06427_gb300 import ks_loop as K
    B, nx = 1216, 64
    u0 = torch.tensor(0.1 * np.random.default_rng(7).standard_normal((B, nx)), device="cuda")
    nsave = args.ncu_dns // 2 + 1
    us = torch.empty(B, nsave, nx, dtype=torch.float64, device="cuda")
    nrm = torch.empty(B, nsave, dtype=torch.float64, device="cuda")
    for _ in range(2):
        K.ks_dns(39.0, nx, B, 0.25, args.ncu_dns, 2, True, u0, us, nrm, None)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_dns": B, "steps": args.ncu_dns}))
    return 0


def ncu_case(args):
    """Small fixed case for ncu captures: set the state, 3 calls of K tau-steps, synchronise."""
    import torch
    from paper_2007_06427_gb300 import ks_loop as K
    from paper_2007_06427_gb300.inputs import workload
    w = workload(args.workload, args.batch)
    mode = K.KS_FP32 if args.mode == "fp32" else K.KS_FP64
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.from_numpy(w.packed()).cuda().to(dt)
    T = torch.tensor(w.T0, dtype=torch.float64, device="cuda")
    with K.KSLoop(w.L, w.nx, w.ns, mode, w.scheme, w.dtau) as h:
        if args.path >= 0:
            K.ks_set_option(h.handle, "path", args.path)
        if args.no_graph:
            K.ks_set_option(h.handle, "graph", 0)
        K.ks_set_state(h.handle, u, T)
        for _ in range(3):
            K.ks_step(h.handle, args.ncu_case, 0.0)
        torch.cuda.synchronize()
    print(json.dumps({"ncu_case": w.name, "mode": args.mode, "steps": 3 * args.ncu_case}))
    return 0


def main():
    args = parse()
    if args.ncu_case:
        return ncu_case(args)
    if args.ncu_dns:
        return ncu_dns(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
