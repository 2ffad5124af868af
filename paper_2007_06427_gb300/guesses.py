"""Initial loops from close recurrences of a chaotic KS run (Sec. 4.3 of the paper).

The paper extracts its initial guesses from a chaotic solution u(x, t) of the KSE: it takes
subsequent maxima of the spatial L2 norm ||u||(t) = (int_0^L u^2 dx)^(1/2) at which
||u||(t + T) ~ ||u||(t), uses the segment between them as the field of the loop and its length
as the period, and removes the high temporal frequencies with a Fourier filter so that the
loop closes smoothly.  This module provides both halves:

* ``ks_dns``: pseudo-spectral time integration of u_t = -u u_x - u_xx - u_xxxx on [0, L)
  (periodic), 2/3-rule dealiasing, fourth-order exponential time differencing (ETDRK4 of Cox &
  Matthews, J. Comput. Phys. 176, 2002, with the phi-functions evaluated by the contour-integral
  average of Kassam & Trefethen, SIAM J. Sci. Comput. 26, 2005);
* ``recurrence_loops``: the recurrence search, segment extraction, temporal low-pass onto the
  descent's band and resampling to Ns points in s.

The paper takes its initial loops from a chaotic run within the subspace of centre-symmetric
fields, u(-x) = -u(x) (Sec. 4.4); ``symmetric=True`` keeps the run there (an odd real field
has purely imaginary Fourier coefficients, and the KSE preserves that, so the projection after
each step only removes rounding).  Every later step of the extraction is linear and acts the
same at x and -x, so the loops it returns are centre-symmetric as well.

Host-side preprocessing (NumPy); the loops it returns are inputs for the GPU descent.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np


def ks_dns(L: float, nx: int, dt: float, nsteps: int, u0: np.ndarray, save_every: int = 1,
           symmetric: bool = False):
    """Integrate the KSE; returns (t [nsave], u [nsave, nx]) sampled every save_every steps.

    symmetric: stay in the centre-symmetric subspace (the real parts of the coefficients are
    zeroed initially and after every step)."""
    k = np.fft.rfftfreq(nx, d=1.0 / nx)                 # 0 .. nx/2
    q = 2.0 * np.pi * k / L
    lin = q ** 2 - q ** 4                               # symbol of -u_xx - u_xxxx
    keep = k <= nx // 3                                 # 2/3 rule
    g = -0.5j * q                                       # N(u) = -(u^2/2)_x
    E = np.exp(dt * lin)
    E2 = np.exp(dt * lin / 2.0)
    # phi-function weights by a contour average around each dt*lin (M points on a circle)
    M = 32
    r = np.exp(1j * np.pi * (np.arange(1, M + 1) - 0.5) / M)
    LR = dt * lin[:, None] + r[None, :]
    Q = dt * np.real(np.mean((np.exp(LR / 2.0) - 1.0) / LR, axis=1))
    f1 = dt * np.real(np.mean((-4.0 - LR + np.exp(LR) * (4.0 - 3.0 * LR + LR ** 2)) / LR ** 3, axis=1))
    f2 = dt * np.real(np.mean((2.0 + LR + np.exp(LR) * (-2.0 + LR)) / LR ** 3, axis=1))
    f3 = dt * np.real(np.mean((-4.0 - 3.0 * LR - LR ** 2 + np.exp(LR) * (4.0 - LR)) / LR ** 3, axis=1))

    def N(vh):
        u = np.fft.irfft(vh, n=nx)
        return g * np.where(keep, np.fft.rfft(u * u), 0.0)

    def sym(vh):
        return 1j * vh.imag if symmetric else vh

    vh = sym(np.where(keep, np.fft.rfft(np.asarray(u0, dtype=np.float64)), 0.0))
    ts, us = [0.0], [np.fft.irfft(vh, n=nx)]
    for n in range(1, nsteps + 1):
        Nv = N(vh)
        a = E2 * vh + Q * Nv
        Na = N(a)
        b = E2 * vh + Q * Na
        Nb = N(b)
        c = E2 * a + Q * (2.0 * Nb - Nv)
        Nc = N(c)
        vh = sym(E * vh + Nv * f1 + 2.0 * (Na + Nb) * f2 + Nc * f3)
        if n % save_every == 0:
            ts.append(n * dt)
            us.append(np.fft.irfft(vh, n=nx))
    return np.asarray(ts), np.asarray(us)


@dataclass
class Guess:
    u: np.ndarray      # [Ns, Nx] loop field on the (x, s) grid, band limited
    T: float           # period (segment length)
    t0: float          # start of the segment in the chaotic run
    mismatch: float    # | ||u||(t0 + T) - ||u||(t0) | / ||u||(t0)


def norm_series(us: np.ndarray, L: float) -> np.ndarray:
    """||u||(t) = (int_0^L u^2 dx)^(1/2) of each saved field (Sec. 4.3)."""
    return np.sqrt(L * np.mean(us * us, axis=1))


def recurrence_loops(ts: np.ndarray, us: np.ndarray, L: float, ns: int,
                     T_range=(10.0, 100.0), tol: float = 0.01, t_min: float = 0.0,
                     max_loops: Optional[int] = None) -> List[Guess]:
    """Loops from subsequent maxima of ||u||(t) with ||u||(t + T) ~ ||u||(t) (Sec. 4.3).

    For every local maximum t_a (after t_min) and every later maximum t_b with T = t_b - t_a in
    T_range and a relative mismatch of the norms below tol, the segment u(., [t_a, t_b)) is
    interpolated to Ns equispaced instants s = n/Ns, Fourier transformed in s, truncated to
    |k| <= Ns/3 (the descent's 2/3 band, which also removes the jump at the closure) and
    transformed back.  Sorted by mismatch, best first."""
    nx = us.shape[1]
    nrm = norm_series(us, L)
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
                cands.append((mis, a, b))
    cands.sort()
    out: List[Guess] = []
    ks = ns // 3
    for mis, a, b in cands:
        T = ts[b] - ts[a]
        s_t = ts[a] + T * np.arange(ns) / ns              # sample instants of the loop
        seg_t = ts[a:b + 1]
        seg = us[a:b + 1]
        loop = np.empty((ns, nx))
        for m in range(nx):                               # linear interpolation in time
            loop[:, m] = np.interp(s_t, seg_t, seg[:, m])
        spec = np.fft.fft(loop, axis=0)
        kk = np.fft.fftfreq(ns, d=1.0 / ns)
        spec[np.abs(kk) > ks, :] = 0.0
        loop = np.real(np.fft.ifft(spec, axis=0))
        # x band as well (the run is dealiased; this only removes the Nyquist mode)
        sx = np.fft.rfft(loop, axis=1)
        sx[:, nx // 3 + 1:] = 0.0
        loop = np.fft.irfft(sx, n=nx, axis=1)
        out.append(Guess(u=loop, T=float(T), t0=float(ts[a]), mismatch=float(mis)))
        if max_loops and len(out) >= max_loops:
            break
    return out


def chaotic_run(L: float, nx: int, t_end: float, dt: float = 0.25, seed: int = 0,
                save_dt: float = 0.5, amplitude: float = 0.1, symmetric: bool = False):
    """A chaotic KS trajectory from a small seeded perturbation (transient included); with
    symmetric, in the centre-symmetric subspace."""
    rng = np.random.default_rng(seed)
    x = L * np.arange(nx) / nx
    u0 = amplitude * (np.cos(2 * np.pi * x / L) * rng.standard_normal()
                      + np.sin(4 * np.pi * x / L) * rng.standard_normal()
                      + 0.3 * rng.standard_normal(nx))
    save_every = max(1, int(round(save_dt / dt)))
    return ks_dns(L, nx, dt, int(round(t_end / dt)), u0, save_every, symmetric=symmetric)
