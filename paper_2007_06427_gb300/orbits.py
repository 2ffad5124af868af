"""Periodic-orbit search at the paper's setting: chaotic run -> recurrence loops -> tau-descent.

The pipeline of Sec. 4.3-4.4: a chaotic KS run in the centre-symmetric subspace, initial loops from
its close recurrences (``guesses.recurrence_loops``), and the descent of all of them together as
one batch on the GPU (mixed precision: float bulk, double finish) with the ``symmetry`` knob set,
so every loop stays in the subspace as the paper's do.  Each converged loop is classified by
what it converged to: the trivial solution u = 0, a steady state (u_s = 0, for which every T is
a fixed point), or a periodic orbit.

    python -m paper_2007_06427_gb300.orbits --L 39 --guesses 8 --max-steps 2000000 --refine-best 2
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import asdict, dataclass
from typing import List, Optional

import numpy as np

from .guesses import Guess, chaotic_run, recurrence_loops


@dataclass
class OrbitResult:
    T0: float             # period of the initial loop (recurrence time)
    t0: float             # start of its segment in the chaotic run
    mismatch: float       # relative norm mismatch of the recurrence
    sqrtJ0: float         # sqrt(J) of the initial loop
    T: float              # final period
    sqrtJ: float          # final sqrt(J)
    steps: int
    status: str
    kind: str             # "trivial", "steady" or "periodic"
    norm: float           # ||u|| = (int int u^2 dx ds)^(1/2) of the final loop
    ds_ratio: float       # ||u_s|| / ||u|| (0 for a steady state)
    refined_steps: int = 0        # steps of the extrapolated refinement (App. C), if any
    extrapolations: int = 0


def classify(u: np.ndarray, L: float, trivial: float = 1e-6, steady: float = 1e-6):
    """(kind, ||u||, ||u_s|| / ||u||) of a loop u[n, m] on the uniform (s, x) grid.

    u_s is the spectral s-derivative (omega_k = 2 pi k); host-side analysis only."""
    ns = u.shape[0]
    norm = math.sqrt(L * float(np.mean(u * u)))
    if norm < trivial:
        return "trivial", norm, 0.0
    uh = np.fft.fft(u, axis=0)
    k = np.fft.fftfreq(ns, d=1.0 / ns)
    us = np.real(np.fft.ifft(2j * np.pi * k[:, None] * uh, axis=0))
    ratio = math.sqrt(L * float(np.mean(us * us))) / norm
    return ("steady" if ratio < steady else "periodic"), norm, ratio


def descend_guesses(guesses: List[Guess], L: float, dtau: float = 0.15, tol: float = 1e-10,
                    max_steps: int = 2_000_000, symmetric: bool = True, mode: str = "mixed",
                    chunk: int = 5000, device: str = "cuda", states: Optional[list] = None,
                    extrapolate: bool = True,
                    extrapolate_start: float = 1e-3) -> List[OrbitResult]:
    """Descend all guesses as one batch (with the extrapolation of App. C inside the descent
    unless extrapolate is False, first anchored once sqrt(J) <= extrapolate_start); returns one
    result per guess (and appends the final loops u[n, m] to ``states`` when given)."""
    import torch
    from . import ks_loop as K
    if not guesses:
        return []
    nx = guesses[0].u.shape[1]
    ns = [g.u.shape[0] for g in guesses]
    kmode = {"mixed": K.KS_MIXED, "fp64": K.KS_FP64, "fp32": K.KS_FP32}[mode]
    B = len(guesses)
    u = torch.from_numpy(np.concatenate([g.u.ravel() for g in guesses])).to(device, torch.float64)
    if kmode == K.KS_FP32:
        u = u.float()
    T = torch.tensor([g.T for g in guesses], dtype=torch.float64, device=device)
    J0 = torch.empty(B, dtype=torch.float64, device=device)
    steps = torch.zeros(B, dtype=torch.int64, device=device)
    sq = torch.zeros(B, dtype=torch.float64, device=device)
    st = torch.zeros(B, dtype=torch.int32, device=device)
    with K.KSLoop(L, nx, ns, kmode, K.KS_IMEX, dtau, tol=tol, max_steps=max_steps,
                  chunk=chunk) as h:
        if symmetric:
            K.ks_set_option(h.handle, "symmetry", 1)
        if extrapolate:
            K.ks_set_option(h.handle, "extrapolate", 1)
            K.ks_set_option(h.handle, "extrapolate_start_ppm", int(round(extrapolate_start * 1e6)))
        K.ks_residual(h.handle, u, T, None, J0)
        K.ks_descend(h.handle, u, T, max_steps, tol, steps, sq, st)
        torch.cuda.synchronize()
    uo = u.double().cpu().numpy()
    out, off = [], 0
    for b, g in enumerate(guesses):
        ub = uo[off:off + ns[b] * nx].reshape(ns[b], nx)
        off += ns[b] * nx
        kind, norm, ratio = classify(ub, L)
        if states is not None:
            states.append(ub.copy())
        out.append(OrbitResult(T0=g.T, t0=g.t0, mismatch=g.mismatch,
                               sqrtJ0=math.sqrt(max(J0[b].item(), 0.0)), T=float(T[b].item()),
                               sqrtJ=float(sq[b].item()), steps=int(steps[b].item()),
                               status=K.STATUS_NAMES.get(int(st[b].item()), str(int(st[b].item()))),
                               kind=kind, norm=norm, ds_ratio=ratio))
    return out


@dataclass
class RefineResult:
    u: np.ndarray         # final loop u[n, m]
    T: float
    steps: int
    sqrtJ: float
    status: int
    extrapolations: int   # moves of App. C kept
    rejected: int         # moves of App. C dropped


def refine(u: np.ndarray, T: float, L: float, dtau: float = 0.15, tol: float = 1e-10,
           max_steps: int = 4_000_000, symmetric: bool = True, device: str = "cuda",
           chunk: int = 5000, switch_tol: float = 1e-5) -> RefineResult:
    """Continue one loop with the mixed-precision descent and the extrapolation of App. C, both
    inside ks_descend (a KS_MIXED handle with the "extrapolate" knob; the float phase ends at
    sqrt(J) = switch_tol, about the float floor, or when sqrt(J) stalls)."""
    import torch
    from . import ks_loop as K
    ns, nx = u.shape
    ut = torch.tensor(u.ravel(), dtype=torch.float64, device=device)
    Tt = torch.tensor([T], dtype=torch.float64, device=device)
    steps = torch.zeros(1, dtype=torch.int64, device=device)
    sq = torch.zeros(1, dtype=torch.float64, device=device)
    st = torch.zeros(1, dtype=torch.int32, device=device)
    with K.KSLoop(L, nx, [ns], K.KS_MIXED, K.KS_IMEX, dtau, tol=tol, switch_tol=switch_tol,
                  max_steps=max_steps, chunk=chunk) as h:
        if symmetric:
            K.ks_set_option(h.handle, "symmetry", 1)
        K.ks_set_option(h.handle, "extrapolate", 1)
        K.ks_descend(h.handle, ut, Tt, max_steps, tol, steps, sq, st)
        kept = K.ks_get_option(h.handle, "extrapolations")
        dropped = K.ks_get_option(h.handle, "extrapolations_rejected")
    return RefineResult(u=ut.cpu().numpy().reshape(ns, nx), T=float(Tt.item()),
                        steps=int(steps.item()), sqrtJ=float(sq.item()), status=int(st.item()),
                        extrapolations=kept, rejected=dropped)


def search(L: float = 39.0, nx: int = 64, ns: int = 64, t_end: float = 3000.0,
           seed: int = 2, guesses: int = 8, T_range=(10.0, 160.0), rec_tol: float = 0.01,
           t_min: float = 200.0, symmetric: bool = True, refine_best: int = 0,
           refine_steps: int = 4_000_000, **descend_kw):
    """The whole pipeline; returns (guesses, results, seconds for the run and the descent).

    refine_best > 0: that many periodic loops with the smallest sqrt(J) that did not
    converge in the batched descent continue alone with the extrapolated mixed descent
    (``refine``)."""
    t0 = time.perf_counter()
    run = chaotic_run(L, nx, t_end, seed=seed, symmetric=symmetric)
    gs = recurrence_loops(run, L, ns, T_range=T_range, tol=rec_tol, t_min=t_min,
                          max_loops=guesses)
    t1 = time.perf_counter()
    states: list = []
    res = descend_guesses(gs, L, symmetric=symmetric, states=states, **descend_kw)
    cand = sorted((i for i, r in enumerate(res) if r.kind == "periodic" and r.status != "converged"),
                  key=lambda i: res[i].sqrtJ)[:refine_best]
    tol = descend_kw.get("tol", 1e-10)
    from . import ks_loop as K
    for i in cand:
        a = refine(states[i], res[i].T, L, tol=tol, max_steps=refine_steps, symmetric=symmetric)
        kind, norm, ratio = classify(a.u, L)
        r = res[i]
        r.refined_steps, r.extrapolations = a.steps, a.extrapolations
        r.T, r.sqrtJ, r.kind, r.norm, r.ds_ratio = a.T, a.sqrtJ, kind, norm, ratio
        r.status = K.STATUS_NAMES.get(int(a.status), str(int(a.status)))
    t2 = time.perf_counter()
    return gs, res, t1 - t0, t2 - t1


def main(argv: Optional[List[str]] = None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--L", type=float, default=39.0)
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--ns", type=int, default=64)
    ap.add_argument("--t-end", type=float, default=3000.0)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--guesses", type=int, default=8)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-steps", type=int, default=2_000_000)
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--no-symmetry", action="store_true")
    ap.add_argument("--refine-best", type=int, default=0,
                    help="continue this many of the best unconverged loops with extrapolation")
    ap.add_argument("--refine-steps", type=int, default=4_000_000)
    ap.add_argument("--extrapolate-start", type=float, default=1e-3,
                    help="sqrt(J) at which the batched descent takes its first extrapolation "
                         "anchor (App. C's example: 1e-3)")
    args = ap.parse_args(argv)
    gs, res, t_guess, t_desc = search(L=args.L, nx=args.nx, ns=args.ns, t_end=args.t_end,
                                      seed=args.seed, guesses=args.guesses,
                                      symmetric=not args.no_symmetry, tol=args.tol,
                                      max_steps=args.max_steps, mode=args.mode,
                                      refine_best=args.refine_best,
                                      refine_steps=args.refine_steps,
                                      extrapolate_start=args.extrapolate_start)
    print(json.dumps({"L": args.L, "nx": args.nx, "ns": args.ns, "guesses": len(gs),
                      "seconds_guesses": t_guess, "seconds_descent": t_desc,
                      "results": [asdict(r) for r in res]}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
