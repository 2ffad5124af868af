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
ks_get_state, ks_residual); the extrapolation itself is one axpy on the host-visible state.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

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


def _sqrtJ(h, u, T):
    J = torch.empty(1, dtype=torch.float64, device=u.device)
    K.ks_residual(h, u, T, None, J)
    return math.sqrt(max(J.item(), 0.0))


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
                         "handle's state would restart its float phase)")
    h = loop.handle
    dev = u.device
    u = u.clone()
    Tt = torch.tensor([T], dtype=torch.float64, device=dev)
    steps_t = torch.zeros(1, dtype=torch.int64, device=dev)
    sq_t = torch.zeros(1, dtype=torch.float64, device=dev)
    st_t = torch.zeros(1, dtype=torch.int32, device=dev)
    K.ks_set_state(h, u, Tt)
    total = 0
    since_set = 0            # the device step counter restarts at every ks_set_state
    anchor = None            # (u, T, sqrtJ) at the start of the current halving segment
    nex = nrej = 0
    hist = []
    status = K.KS_RUNNING
    sq = _sqrtJ(h, u, Tt)
    while total < max_steps:
        if sq < tol:
            status = K.KS_CONVERGED
            break
        n = min(chunk, max_steps - total)
        K.ks_step(h, n, tol)
        K.ks_get_state(h, u, Tt, steps_t, sq_t, st_t)
        total += int(steps_t.item()) - since_set
        since_set = int(steps_t.item())
        sq = _sqrtJ(h, u, Tt)
        hist.append((total, sq, "step"))
        if int(st_t.item()) not in (K.KS_RUNNING, K.KS_CONVERGED):
            status = int(st_t.item())
            break
        if sq < tol:
            status = K.KS_CONVERGED
            break
        if sq > start:
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
        sqe = _sqrtJ(h, ue, Te)
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
    else:
        status = K.KS_STEP_CAP
    return AccelResult(u=u, T=float(Tt.item()), steps=total, sqrtJ=sq, status=status,
                       extrapolations=nex, rejected=nrej, history=hist)
