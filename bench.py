#!/usr/bin/env python
"""Benchmark of the KS loop tau-descent on GB300: tau-step gridpoints/s and (unless --no-to-tol)
wall time to sqrt(J) < 1e-10 for plain FP64 against FP32-bulk + FP64-finish, plus the FP64
descent with the extrapolation of App. C.

One bench step is one tau-step of the whole hot path (residual, reductions, adjoint, update)
over the workload's batch, on the resident state in HBM.  The L2 cache is flushed (a 256 MiB
write) before every timed step and each step is timed with CUDA events on the launch stream.
Under torchrun every rank descends its own seeded loops (weak scaling, no collective on the
data path); the reported time is the max over ranks.

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
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
                    help="skip the FP64 vs mixed descent to sqrt(J) < tol")
    ap.add_argument("--no-fp32", action="store_true", help="skip the float-path throughput line")
    ap.add_argument("--to-tol-max-steps", type=int, default=1_000_000)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--switch-tol", type=float, default=0.0,
                    help="mixed: switch to double once sqrt(J) (evaluated in double) <= this; "
                         "0: switch when it stops falling over the stall window")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="K",
                    help="profiling case: load the workload, run 3 x K tau-steps, no timing")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
# algorithmic work per launch (FFT counted as 5 n log2 n flops per complex transform)
# ---------------------------------------------------------------------------------------
def fft_flops(n: int) -> float:
    return 5.0 * n * math.log2(n)


def kernel_flops(kind: str, nx: int, nss, steps_per_launch: int = 1) -> float:
    """Algorithmic flops of one launch of `kind` over the batch.

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


def measured_traffic(workload: str, kernel: str):
    """DRAM bytes per launch from the committed ncu capture, if the CUDA sources still match."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_sha") != kernel_source_hash():
        return None
    e = t.get("kernels", {}).get(f"{workload}/{kernel}")
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
        "config": {"workload": args.workload, "L": w.L, "nx": w.nx, "ns": w.ns[:8],
                   "batch": w.batch, "scheme": "imex" if w.scheme else "explicit",
                   "dtau": w.dtau},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{r['steps']} oracle tau-steps of the workload (NumPy FP64 "
                                   "dense DFTs, single-threaded BLAS)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ours_arm(args):
    import numpy as np
    import torch
    from paper_2007_06427_gb300 import ks_loop as K
    from paper_2007_06427_gb300.inputs import workload

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

    w = workload(args.workload, args.batch)
    if ws > 1:
        # every rank descends its own loops: seeds offset by rank
        from paper_2007_06427_gb300.inputs import make_loops
        base = workload(args.workload, args.batch)
        w = make_loops(base.name, base.nx, base.L, [rank * base.batch + i for i in range(base.batch)],
                       ns=base.ns[0] if len(set(base.ns)) == 1 else None,
                       ns_choices=None if len(set(base.ns)) == 1 else (32, 64, 128, 256),
                       T_range=(20.0, 80.0), scheme=base.scheme, dtau=base.dtau)
    mode = K.KS_FP32 if args.mode == "fp32" else K.KS_FP64
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    nx, nss = w.nx, w.ns
    gp = w.gridpoints
    stream = torch.cuda.current_stream(dev)
    u = torch.from_numpy(w.packed()).to(dev, dt)
    T = torch.tensor(w.T0, dtype=torch.float64, device=dev)
    h = K.KSLoop(w.L, nx, nss, mode, w.scheme, w.dtau, autotune=int(args.autotune))
    K.ks_set_state(h.handle, u, T, stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    for _ in range(args.warmup):
        K.ks_step(h.handle, 1, 0.0, stream)
    torch.cuda.synchronize(dev)
    prof, per_step = profile_pass(K, h, args, flush, stream, dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(lrank)
    clk.start()
    evs = []
    for _ in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.ks_step(h.handle, 1, 0.0, stream)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clocks = clk.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = int(round(per_step * args.steps))
    tmax = total_ms
    if pg:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        tmax = float(t.item())
    value = ws * gp * args.steps / (tmax / 1e3)

    roof = annotate_sms(roofline_entry(prof, total_ms / args.steps, w, nx, nss), K, h, mode,
                        w.batch, dev)

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
        e2e = {"value": ws * gp * E * args.e2e_calls / el, "unit": UNIT,
               "h2d_bytes_per_step": ub + 8 * w.batch,
               "d2h_bytes_per_step": ub + (8 + 8 + 8 + 4) * w.batch,
               "tau_steps_per_call": E,
               "note": "one bench step = one ks_descend call on pinned host buffers"}

    to_tol = None
    if not args.no_to_tol and ws == 1:
        to_tol = run_to_tol(args, w, dev)

    fp32 = None
    if not args.no_fp32 and mode == K.KS_FP64:
        fp32 = throughput_fp32(args, w, dev, flush, K)

    launch_shape = {"path": K.ks_get_option(h.handle, "path"),
                    "cluster": K.ks_get_option(h.handle, "cluster_f32" if mode == K.KS_FP32 else "cluster_f64"),
                    "threads": K.ks_get_option(h.handle, "cluster_threads"),
                    "autotuned": bool(args.autotune)}
    h.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if mode == K.KS_FP32 else "f64", "data": "synthetic",
            "config": {"workload": w.name, "L": w.L, "nx": nx, "ns": nss[:8], "batch": w.batch,
                       "scheme": "imex" if w.scheme else "explicit", "dtau": w.dtau,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "gridpoints": gp,
                       "launch": launch_shape},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "kernels_profiled_pass": {"steps": PROFILE_STEPS,
                                      **{k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}},
        }
        if to_tol:
            if cpu and cpu.get("value"):
                # the oracle at the measured per-step rate for the same step counts (FP64 runs)
                for key in ("fp64", "fp64_extrapolated"):
                    if key in to_tol:
                        n = sum(to_tol[key]["steps"]) if w.batch == 1 else to_tol[key]["steps"][0]
                        to_tol[key]["cpu_oracle_seconds_extrapolated"] = n * w.gridpoints / cpu["value"]
            # the whole descent against the roofline: algorithmic flops of its steps over its
            # wall time (read-backs, monitors and extrapolations included); FP64 runs against
            # the FP64 peak, mixed runs (mostly FP32 steps) reported as achieved only
            # flops per loop-step (mean over the batch; exact for a single loop or equal Ns)
            fl = step_flops(nx, nss) / w.batch
            for key, v in to_tol.items():
                if isinstance(v, dict) and v.get("seconds") and len(set(nss)) == 1:
                    ach = fl * v["total_steps"] / v["seconds"] / 1e12
                    v["achieved_tflops"] = ach
                    if key.startswith("fp64"):
                        v["frac_of_fp64_peak"] = ach / PEAK_TFLOPS["f64"]
            line["time_to_tol"] = to_tol
        if fp32:
            line["fp32"] = fp32
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


PROFILE_STEPS = 20


def profile_pass(K, h, args, flush, stream, dev, nsteps: int = PROFILE_STEPS):
    """An untimed pass of nsteps bench steps (same pattern: flush, one ks_step) with the
    library's per-kernel event timing on.  Returns ({kind: (ms, launches)}, launches per step).
    The timed region runs without the library's own events, which would add device work to
    every step."""
    import torch
    K.ks_profile(h.handle, True)
    K.ks_profile_read(h.handle, reset=True)
    for _ in range(nsteps):
        if not args.no_flush:
            flush.zero_()
        K.ks_step(h.handle, 1, 0.0, stream)
    torch.cuda.synchronize(dev)
    prof, launches = K.ks_profile_read(h.handle, reset=True)
    K.ks_profile(h.handle, False)
    return prof, launches / nsteps


def roofline_entry(prof, ms_per_step, w, nx, nss):
    """Roofline of the dominant kernel: its launch duration is the timed region's mean step time
    (CUDA events on the launch stream) times the kernel's share of the library's device time in
    the profiled pass, per launch."""
    dname = max(prof, key=lambda k: prof[k][0]) if prof else None
    if not dname:
        return None
    ms_k, cnt = prof[dname]
    tot = max(sum(v[0] for v in prof.values()), 1e-30)
    share = ms_k / tot
    launches_per_step = cnt / PROFILE_STEPS
    ms_launch = ms_per_step * share / max(launches_per_step, 1e-30)
    fl = kernel_flops(dname, nx, nss)
    ach = fl / (ms_launch / 1e3) / 1e12 if ms_launch > 0 else 0.0
    pk = PEAK_TFLOPS["f32" if dname.endswith("f32") else "f64"]
    return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
            "frac": ach / pk, "traffic": measured_traffic(w.name, dname), "kernel": dname,
            "flops_per_launch": fl, "ms_per_launch": ms_launch,
            "ms_per_launch_profiled": ms_k / cnt, "share": share,
            "peak_source": ("nominal GB300 FP64 rate (1.25 TFLOP/s)" if not dname.endswith("f32")
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


def throughput_fp32(args, w, dev, flush, K):
    """Same timed loop on an FP32 handle (the bulk phase of a mixed descent)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    u = torch.from_numpy(w.packed()).to(dev, torch.float32)
    T = torch.tensor(w.T0, dtype=torch.float64, device=dev)
    h = K.KSLoop(w.L, w.nx, w.ns, K.KS_FP32, w.scheme, w.dtau, autotune=int(args.autotune))
    K.ks_set_state(h.handle, u, T, stream)
    for _ in range(args.warmup):
        K.ks_step(h.handle, 1, 0.0, stream)
    torch.cuda.synchronize(dev)
    prof, per_step = profile_pass(K, h, args, flush, stream, dev)
    evs = []
    for _ in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.ks_step(h.handle, 1, 0.0, stream)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    out = {"value": w.gridpoints * args.steps / (total_ms / 1e3), "unit": UNIT,
           "ms_per_step": total_ms / args.steps, "dtype": "f32",
           "gpu_launches": int(round(per_step * args.steps))}
    roof = annotate_sms(roofline_entry(prof, total_ms / args.steps, w, w.nx, w.ns), K, h,
                        K.KS_FP32, w.batch, dev)
    h.close()
    if roof:
        out["roofline"] = roof
    return out


def outcome_counts(K, st):
    """Loops of the batch per final status (converged, step cap, stalled, diverged)."""
    out = {}
    for v in st.tolist():
        name = K.STATUS_NAMES.get(int(v), str(int(v)))
        out[name] = out.get(name, 0) + 1
    return out


def run_to_tol(args, w, dev):
    """Plain FP64 descent vs FP32 bulk + FP64 finish, from the same loops, to sqrt(J) < tol;
    then both again with the extrapolation of App. C inside ks_descend."""
    import numpy as np
    import torch
    from paper_2007_06427_gb300 import ks_loop as K
    out = {}
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    clk.start()
    for name, mode in (("fp64", K.KS_FP64), ("mixed", K.KS_MIXED)):
        h = K.KSLoop(w.L, w.nx, w.ns, mode, w.scheme, w.dtau, tol=args.tol,
                     switch_tol=args.switch_tol, max_steps=args.to_tol_max_steps, chunk=2000)
        u = torch.from_numpy(w.packed()).to(dev, torch.float64)
        T = torch.tensor(w.T0, dtype=torch.float64, device=dev)
        steps = torch.zeros(w.batch, dtype=torch.int64, device=dev)
        sq = torch.zeros(w.batch, dtype=torch.float64, device=dev)
        st = torch.zeros(w.batch, dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        K.ks_descend(h.handle, u, T, args.to_tol_max_steps, args.tol, steps, sq, st)
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        hs, hq, hp = K.ks_get_history(h.handle, 0)
        marks = {}
        for target in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10):
            idx = np.nonzero(hq < target)[0]
            if idx.size:
                marks[f"{target:.0e}"] = int(hs[idx[0]])
        switch = int(hs[np.nonzero(hp == 0)[0][0]]) if (name == "mixed" and (hp == 0).any()) else None
        out[name] = {"seconds": el, "steps": steps.tolist()[:8], "sqrtJ": sq.tolist()[:8],
                     "status": [K.STATUS_NAMES.get(int(s), str(int(s))) for s in st.tolist()[:8]],
                     "outcomes": outcome_counts(K, st), "total_steps": int(steps.sum().item()),
                     "T": T.tolist()[:8], "loop0_first_step_below": marks,
                     "loop0_switch_step": switch,
                     "loop0_history": [[int(a), float(c)] for a, c in zip(hs[::max(1, len(hs) // 40)], hq[::max(1, len(hq) // 40)])]}
        h.close()
    # the same two descents with the extrapolation of App. C inside ks_descend
    # (the extrapolated mixed run switches to double at sqrt(J) = 1e-5, about the float floor of
    # this loop: the jumps of the extrapolation restart the stall window the plain run waits on)
    for name, mode in (("fp64_extrapolated", K.KS_FP64), ("mixed_extrapolated", K.KS_MIXED)):
        sw = max(args.switch_tol, 1e-5) if mode == K.KS_MIXED else 0.0
        h = K.KSLoop(w.L, w.nx, w.ns, mode, w.scheme, w.dtau, tol=args.tol,
                     switch_tol=sw, max_steps=args.to_tol_max_steps, chunk=1000)
        K.ks_set_option(h.handle, "extrapolate", 1)
        u = torch.from_numpy(w.packed()).to(dev, torch.float64)
        T = torch.tensor(w.T0, dtype=torch.float64, device=dev)
        steps = torch.zeros(w.batch, dtype=torch.int64, device=dev)
        sq = torch.zeros(w.batch, dtype=torch.float64, device=dev)
        st = torch.zeros(w.batch, dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        K.ks_descend(h.handle, u, T, args.to_tol_max_steps, args.tol, steps, sq, st)
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        hs, hq, hp = K.ks_get_history(h.handle, 0)
        switch = int(hs[np.nonzero(hp == 0)[0][0]]) if (mode == K.KS_MIXED and (hp == 0).any()) else None
        out[name] = {"seconds": el, "steps": steps.tolist()[:8], "sqrtJ": sq.tolist()[:8],
                     "status": [K.STATUS_NAMES.get(int(v), str(int(v))) for v in st.tolist()[:8]],
                     "outcomes": outcome_counts(K, st), "total_steps": int(steps.sum().item()),
                     "T": T.tolist()[:8],
                     "extrapolations": K.ks_get_option(h.handle, "extrapolations"),
                     "rejected": K.ks_get_option(h.handle, "extrapolations_rejected"),
                     "loop0_switch_step": switch, "switch_tol": sw,
                     "note": "App. C inside ks_descend: from sqrt(J) = 1e-3, geometric extrapolation "
                             "each time sqrt(J) (evaluated in double every 1000 steps) halves"}
        h.close()
    out["clocks"] = clk.stop()
    return out


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
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
