"""Acceleration of the tau-descent by linear extrapolation (App. C of the paper).

Near an attracting fixed point l* the descent approaches along the leading eigendirection of
the linearised loop dynamics: l(tau) - l* ~ c v exp(-lambda tau), so sqrt(J) is proportional
to |l - l*|.  The paper integrates until sqrt(J) = 1e-3, then repeatedly integrates until
sqrt(J) has halved and extrapolates along the trajectory.  It gives no formula; the reading used
here is geometric extrapolation from the two states at either end of a halving segment:

    rho = sqrt(J_b) / sqrt(J_a),   l* ~ l_b + (l_b - l_a) rho / (1 - rho)

applied to both u (on the grid; the map is linear, so this equals extrapolating the band state)
and T.  An extrapolated loop whose sqrt(J) is not below sqrt(J_b) is rejected and the descent
continues from l_b, so sqrt(J) never increases.

Runs on the GPU through the resident-state calls of the C ABI (ks_set_state, ks_step,
ks_get_state, ks_residual); the extrapolation itself is one axpy on the device-resident state.
``descend_extrapolated`` works on a double handle; ``descend_extrapolated_mixed`` runs the same
scheme on a float handle until sqrt(J), evaluated in double, reaches the float floor or stalls,
and finishes on a double handle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import torch

from . import ks_loop as K


@dataclass
class AccelResult:
    u: torch.Tensor
    T: float
    steps: int
    sqrtJ: float
    status: int
    extrapolations: int
    rejected: int
    history: List[tuple] = field(default_factory=list)   # (steps, sqrtJ, event)
    switch_step: Optional[int] = None                     # mixed: first double step


def _sqrtJ(h, u, T):
    J = torch.empty(1, dtype=torch.float64, device=u.device)
    K.ks_residual(h, u, T, None, J)
    return math.sqrt(max(J.item(), 0.0))


def _core(h, u: torch.Tensor, Tt: torch.Tensor, sqrtJ_of: Callable, tol: float, max_steps: int,
          start: float, drop: float, chunk: int, total0: int, hist: list,
          leave: Optional[Callable] = None):
    """The extrapolated descent of one loop on handle h (state u, Tt already resident).

    Returns (u, Tt, sqrtJ, steps, status, extrapolations, rejected, left); ``left`` is True when
    ``leave(sqrtJ, steps)`` asked to stop (the float phase of a mixed descent)."""
    dev = u.device
    steps_t = torch.zeros(1, dtype=torch.int64, device=dev)
    sq_t = torch.zeros(1, dtype=torch.float64, device=dev)
    st_t = torch.zeros(1, dtype=torch.int32, device=dev)
    total = total0
    since_set = 0            # the device step counter restarts at every ks_set_state
    anchor = None            # (u, T, sqrtJ) at the start of the current halving segment
    nex = nrej = 0
    sq = sqrtJ_of(u, Tt)
    while total < max_steps:
        if sq < tol:
            return u, Tt, sq, total, K.KS_CONVERGED, nex, nrej, False
        if leave is not None and leave(sq, total):
            return u, Tt, sq, total, K.KS_RUNNING, nex, nrej, True
        n = min(chunk, max_steps - total)
        K.ks_step(h, n, 0.0)
        K.ks_get_state(h, u, Tt, steps_t, sq_t, st_t)
        total += int(steps_t.item()) - since_set
        since_set = int(steps_t.item())
        sq = sqrtJ_of(u, Tt)
        hist.append((total, sq, "step"))
        if int(st_t.item()) not in (K.KS_RUNNING, K.KS_CONVERGED):
            return u, Tt, sq, total, int(st_t.item()), nex, nrej, False
        if sq < tol or sq > start:
            continue
        if anchor is None:
            anchor = (u.clone(), Tt.clone(), sq)
            continue
        if sq > drop * anchor[2]:
            continue
        # extrapolate from the halving segment [anchor, now]
        rho = sq / anchor[2]
        c = rho / (1.0 - rho)
        ue = u + (u - anchor[0]) * c
        Te = Tt + (Tt - anchor[1]) * c
        sqe = sqrtJ_of(ue, Te)
        if sqe < sq:
            u, Tt, sq = ue, Te, sqe
            nex += 1
            hist.append((total, sq, "extrapolated"))
        else:
            nrej += 1
            hist.append((total, sqe, "rejected"))
        anchor = (u.clone(), Tt.clone(), sq)
        K.ks_set_state(h, u, Tt)
        since_set = 0
    return u, Tt, sq, total, (K.KS_CONVERGED if sq < tol else K.KS_STEP_CAP), nex, nrej, False


def descend_extrapolated(loop: "K.KSLoop", u: torch.Tensor, T: float, tol: float = 1e-10,
                         max_steps: int = 1_000_000, start: float = 1e-3,
                         drop: float = 0.5, chunk: int = 200) -> AccelResult:
    """Tau-descent of ONE loop (batch 1 handle, double state) with extrapolation.

    u: device tensor (the handle's element type), T: period.  Integrates in chunks of `chunk`
    steps; from sqrt(J) <= start on, every time sqrt(J) has fallen by the factor `drop` since
    the last anchor it extrapolates (App. C reading above)."""
    if loop.batch != 1:
        raise ValueError("descend_extrapolated works on a single-loop handle")
    if loop.mode != K.KS_FP64:
        raise ValueError("descend_extrapolated needs a KS_FP64 handle (re-setting a mixed "
                         "handle's state would restart its float phase); use "
                         "descend_extrapolated_mixed for a float bulk")
    h = loop.handle
    u = u.clone()
    Tt = torch.tensor([T], dtype=torch.float64, device=u.device)
    K.ks_set_state(h, u, Tt)
    hist: list = []
    u, Tt, sq, total, status, nex, nrej, _ = _core(
        h, u, Tt, lambda a, b: _sqrtJ(h, a, b), tol, max_steps, start, drop, chunk, 0, hist)
    return AccelResult(u=u, T=float(Tt.item()), steps=total, sqrtJ=sq, status=status,
                       extrapolations=nex, rejected=nrej, history=hist)


def descend_extrapolated_mixed(loop32: "K.KSLoop", loop64: "K.KSLoop", u: torch.Tensor,
                               T: float, tol: float = 1e-10, max_steps: int = 1_000_000,
                               switch_tol: float = 1e-5, stall_window: int = 40_000,
                               stall_drop: float = 1e-3, start: float = 1e-3,
                               drop: float = 0.5, chunk: int = 1000) -> AccelResult:
    """Extrapolated descent with a float bulk and a double finish (one loop).

    loop32: a KS_FP32 handle, loop64: a KS_FP64 handle of the same loop shape.  The float phase
    evaluates sqrt(J) in double (loop64's residual of the widened state) and hands over to the
    double phase once that value is <= switch_tol or has not fallen by the fraction stall_drop
    within stall_window steps (the float rounding floor); both phases extrapolate."""
    if loop32.batch != 1 or loop64.batch != 1:
        raise ValueError("descend_extrapolated_mixed works on single-loop handles")
    if loop32.mode != K.KS_FP32 or loop64.mode != K.KS_FP64:
        raise ValueError("descend_extrapolated_mixed needs a KS_FP32 and a KS_FP64 handle")
    h32, h64 = loop32.handle, loop64.handle
    dev = u.device
    u32 = u.to(torch.float32).clone()
    Tt = torch.tensor([T], dtype=torch.float64, device=dev)
    K.ks_set_state(h32, u32, Tt)
    hist: list = []
    best = [float("inf"), 0]           # best sqrt(J) so far and the step it was reached

    def leave(sq, total):
        if sq <= switch_tol:
            return True
        if sq < (1.0 - stall_drop) * best[0]:
            best[0], best[1] = sq, total
        return total - best[1] >= stall_window

    def sqrtJ_f32(a, b):
        return _sqrtJ(h64, a.to(torch.float64), b)

    u32, Tt, sq, total, status, nex, nrej, left = _core(
        h32, u32, Tt, sqrtJ_f32, tol, max_steps, start, drop, chunk, 0, hist, leave)
    if not left:
        return AccelResult(u=u32.to(torch.float64), T=float(Tt.item()), steps=total, sqrtJ=sq,
                           status=status, extrapolations=nex, rejected=nrej, history=hist)
    switch = total
    hist.append((total, sq, "switch"))
    u64 = u32.to(torch.float64)
    K.ks_set_state(h64, u64, Tt)
    u64, Tt, sq, total, status, nex2, nrej2, _ = _core(
        h64, u64, Tt, lambda a, b: _sqrtJ(h64, a, b), tol, max_steps, start, drop, chunk,
        total, hist)
    return AccelResult(u=u64, T=float(Tt.item()), steps=total, sqrtJ=sq, status=status,
                       extrapolations=nex + nex2, rejected=nrej + nrej2, history=hist,
                       switch_step=switch)
