"""Initial loops from close recurrences of a chaotic KS run (Sec. 4.3 of the paper).

The paper extracts its initial guesses from a chaotic solution u(x, t) of the KSE: it takes
subsequent maxima of the spatial L2 norm ||u||(t) = (int_0^L u^2 dx)^(1/2) at which
||u||(t + T) ~ ||u||(t), uses the segment between them as the field of the loop and its length
as the period, and removes the high temporal frequencies with a Fourier filter so that the
loop closes smoothly.  Both halves run on the GPU through the C ABI:

* ``ks_dns``: the run itself (``ks_dns`` in the library: Fourier pseudo-spectral in x, 2/3-rule
  dealiasing, fourth-order exponential time differencing), which also returns ||u||(t) at every
  saved instant;
* ``recurrence_loops``: the recurrence search over the norm series (``recurrence_pairs``, index
  bookkeeping on the host), the segment cut to Ns instants by linear interpolation in time
  (``ks_dns_segments``) and the temporal low-pass, which is the projection onto the descent's
  2/3 band (|k| <= Ns/3, which also removes the jump at the closure, and |j| <= Nx/3) that a
  loop handle applies to every input (``ks_set_state`` / ``ks_get_state``).

The paper takes its initial loops from a chaotic run within the subspace of centre-symmetric
fields, u(-x) = -u(x) (Sec. 4.4); ``symmetric=True`` keeps the run there (an odd real field
has purely imaginary Fourier coefficients, and the KSE preserves that, so the projection after
each step only removes rounding).  Every later step of the extraction is linear and acts the
same at x and -x, so the loops it returns are centre-symmetric as well.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, NamedTuple, Optional

import numpy as np

from . import ks_loop as K


class Run(NamedTuple):
    ts: np.ndarray    # [nsave] saved instants, t = 0 first
    us: "object"      # torch tensor on the device, [nsave, nx] (or [batch, nsave, nx])
    norms: np.ndarray  # ||u||(t) at the saved instants, [nsave] (or [batch, nsave])


def ks_dns(L: float, nx: int, dt: float, nsteps: int, u0, save_every: int = 1,
           symmetric: bool = False, device: str = "cuda") -> Run:
    """Integrate the KSE on the GPU from the grid field(s) u0 ([nx] or [batch, nx]); the state is
    saved every save_every steps (t = 0 first).  symmetric: stay in the centre-symmetric
    subspace (the real parts of the coefficients are zeroed initially and after every step)."""
    import torch
    u0 = torch.as_tensor(np.asarray(u0, dtype=np.float64)).to(device)
    single = u0.dim() == 1
    u0 = u0.reshape(-1, nx).contiguous()
    batch = u0.shape[0]
    nsave = nsteps // save_every + 1
    us = torch.empty(batch, nsave, nx, dtype=torch.float64, device=device)
    norms = torch.empty(batch, nsave, dtype=torch.float64, device=device)
    with torch.cuda.device(u0.device):
        K.ks_dns(L, nx, batch, dt, nsteps, save_every, symmetric, u0, us, norms,
                 stream=torch.cuda.current_stream())
    ts = dt * save_every * np.arange(nsave, dtype=np.float64)
    nrm = norms.cpu().numpy()
    if single:
        return Run(ts, us[0], nrm[0])
    return Run(ts, us, nrm)


@dataclass
class Guess:
    u: np.ndarray      # [Ns, Nx] loop field on the (x, s) grid, band limited
    T: float           # period (segment length)
    t0: float          # start of the segment in the chaotic run
    mismatch: float    # | ||u||(t0 + T) - ||u||(t0) | / ||u||(t0)


def recurrence_pairs(ts: np.ndarray, norms: np.ndarray, T_range=(10.0, 100.0), tol: float = 0.01,
                     t_min: float = 0.0):
    """Close recurrences of a norm series (Sec. 4.3): every pair of local maxima t_a < t_b of
    ||u||(t) (t_a >= t_min) with T = t_b - t_a in T_range and a relative mismatch
    | ||u||(t_b) - ||u||(t_a) | / ||u||(t_a) below tol, as (mismatch, a, b) sorted best first."""
    nrm = np.asarray(norms)
    idx = [i for i in range(1, len(nrm) - 1)
           if nrm[i] > nrm[i - 1] and nrm[i] >= nrm[i + 1] and ts[i] >= t_min]
    cands = []
    for a_i, a in enumerate(idx):
        for b in idx[a_i + 1:]:
            T = ts[b] - ts[a]
            if T < T_range[0]:
                continue
            if T > T_range[1]:
                break
            mis = abs(nrm[b] - nrm[a]) / nrm[a]
            if mis < tol:
                cands.append((float(mis), a, b))
    cands.sort()
    return cands


def recurrence_loops(run: Run, L: float, ns: int, T_range=(10.0, 100.0), tol: float = 0.01,
                     t_min: float = 0.0, max_loops: Optional[int] = None) -> List[Guess]:
    """Loops from the close recurrences of one saved run (``recurrence_pairs``): the segment
    u(., [t_a, t_b)) at Ns equispaced instants s = n/Ns (linear interpolation in time, on the
    GPU), projected onto the descent's 2/3 band |j| <= Nx/3, |k| <= Ns/3 (the temporal low-pass
    of Sec. 4.3), returned on the grid.  Sorted by mismatch, best first."""
    import torch
    ts, us, nrm = run
    cands = recurrence_pairs(ts, nrm, T_range, tol, t_min)
    if max_loops:
        cands = cands[:max_loops]
    if not cands:
        return []
    nsave, nx = us.shape
    dts = float(ts[1] - ts[0])
    a_idx = np.array([a for _, a, _ in cands], dtype=np.int32)
    Ts = np.array([ts[b] - ts[a] for _, a, b in cands], dtype=np.float64)
    B = len(cands)
    dev = us.device
    raw = torch.empty(B * ns * nx, dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream()
        K.ks_dns_segments(nx, nsave, dts, us.contiguous(), a_idx, Ts, [ns] * B, raw, stream=stream)
        out = torch.empty_like(raw)
        Tt = torch.tensor(Ts, dtype=torch.float64, device=dev)
        with K.KSLoop(L, nx, [ns] * B, K.KS_FP64) as h:
            K.ks_set_state(h.handle, raw, Tt, stream=stream)
            K.ks_get_state(h.handle, out, stream=stream)
        torch.cuda.synchronize(dev)
    loops = out.cpu().numpy().reshape(B, ns, nx)
    return [Guess(u=loops[i], T=float(Ts[i]), t0=float(ts[a]), mismatch=float(mis))
            for i, (mis, a, _) in enumerate(cands)]


def chaotic_run(L: float, nx: int, t_end: float, dt: float = 0.25, seed: int = 0,
                save_dt: float = 0.5, amplitude: float = 0.1, symmetric: bool = False,
                device: str = "cuda") -> Run:
    """A chaotic KS trajectory from a small seeded perturbation (transient included); with
    symmetric, in the centre-symmetric subspace."""
    rng = np.random.default_rng(seed)
    x = L * np.arange(nx) / nx
    u0 = amplitude * (np.cos(2 * np.pi * x / L) * rng.standard_normal()
                      + np.sin(4 * np.pi * x / L) * rng.standard_normal()
                      + 0.3 * rng.standard_normal(nx))
    save_every = max(1, int(round(save_dt / dt)))
    return ks_dns(L, nx, dt, int(round(t_end / dt)), u0, save_every, symmetric=symmetric,
                  device=device)
