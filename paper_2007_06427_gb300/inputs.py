"""Seeded synthetic loops for the KS tau-descent workloads.

This module only draws inputs; it holds none of the descent's arithmetic.  Both the CUDA
path's tests/benchmarks and the CPU oracle's tests take their inputs from here.

Recipe (per loop b, generator ``numpy.random.default_rng(seed_b)``, draws in this order):

1. if the workload gives a set of N_s values, ``N_s = rng.choice(set)``;
2. if the workload gives a period range, ``T0 = rng.uniform(lo, hi)``, else T0 is fixed;
3. ``re, im = rng.standard_normal((Kx+1, 2Ks+1))`` twice, for the half-spectrum modes
   j = 0..Kx, k = -Ks..Ks of the 2/3 band (Kx = N_x // 3, Ks = N_s // 3);
4. coefficient c_jk = (re + i im) * exp(-|j| / d_x) * exp(-|k| / d_s); the j = 0 column is
   set to zero (zero spatial mean); modes with j < 0 are the complex conjugates
   c_{-j,-k} = conj(c_{j,k}) so the field is real;
5. u(x_m, s_n) = sum_jk c_jk exp(2 pi i (m j / N_x + n k / N_s)), then u is scaled so that its
   grid rms is 1.

Centre-symmetric loops (``symmetric=True``, the subspace the paper's orbits lie in, Sec. 4.4):
same draws, then c_jk <- (c_jk - conj(c_{j,-k})) / 2 before step 5, which makes u odd in x,
u(-x, s) = -u(x, s).

The loops are band limited by construction, so the 2/3-rule projection leaves them unchanged
up to rounding.  The paper draws its initial loops from recurrences of a chaotic KS run
(Sec. 4.3); these seeded spectral loops stand in for that data, which is not available.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclass
class Workload:
    name: str
    L: float
    nx: int
    ns: List[int]
    T0: List[float]
    u: List[np.ndarray]          # grid fields u[n, m], float64
    scheme: int                  # 0 explicit, 1 IMEX
    dtau: float
    meta: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return len(self.ns)

    @property
    def gridpoints(self) -> int:
        return int(sum(n * self.nx for n in self.ns))

    def packed(self) -> np.ndarray:
        """Ragged-packed [sum_b Ns_b * Nx] float64 array, loop-major, m fastest."""
        return np.concatenate([a.reshape(-1) for a in self.u]) if self.u else np.zeros(0)


def spectral_loop(seed: int, nx: int, L: float, ns: Optional[int] = None,
                  ns_choices: Optional[Sequence[int]] = None, T0: Optional[float] = None,
                  T_range: Optional[Tuple[float, float]] = None, decay=(2.0, 2.0),
                  rms: float = 1.0, symmetric: bool = False):
    """One seeded loop (u grid [Ns, Nx] float64, T0, Ns) following the module recipe."""
    rng = np.random.default_rng(seed)
    if ns_choices is not None:
        ns = int(rng.choice(np.asarray(ns_choices)))
    if ns is None:
        raise ValueError("give ns or ns_choices")
    if T_range is not None:
        T = float(rng.uniform(T_range[0], T_range[1]))
    else:
        T = float(T0)
    kx, ks = nx // 3, ns // 3
    re = rng.standard_normal((kx + 1, 2 * ks + 1))
    im = rng.standard_normal((kx + 1, 2 * ks + 1))
    j = np.arange(kx + 1)
    k = np.arange(-ks, ks + 1)
    amp = np.exp(-j / decay[0])[:, None] * np.exp(-np.abs(k) / decay[1])[None, :]
    c = (re + 1j * im) * amp
    c[0, :] = 0.0
    if symmetric:
        c = 0.5 * (c - np.conj(c[:, ::-1]))       # column k = -Ks..Ks reversed is -k
    # real synthesis: u = 2 Re sum_{j>=1} sum_k c_jk e^{2 pi i (m j / Nx + n k / Ns)}
    m = np.arange(nx)
    n = np.arange(ns)
    ex = np.exp(2j * np.pi * np.outer(j, m) / nx)          # [j, m]
    es = np.exp(2j * np.pi * np.outer(n, k) / ns)          # [n, k]
    u = 2.0 * (es @ c.T @ ex).real                          # [n, m]
    s = float(np.sqrt(np.mean(u * u)))
    if s > 0:
        u *= rms / s
    return u, T, ns


def with_white_noise(u: np.ndarray, seed: int, amp: float = 0.5) -> np.ndarray:
    """u plus seeded white noise of grid rms ``amp``: energy in every Fourier mode of the grid,
    inside and outside the 2/3 band, the Nyquist modes included (generator
    ``numpy.random.default_rng(10_000 + seed)``)."""
    rng = np.random.default_rng(10_000 + seed)
    return u + amp * rng.standard_normal(u.shape)


def outside_band_modes(nx: int, ns: int, amp: float = 1.0) -> np.ndarray:
    """A real grid field [Ns, Nx] made only of Fourier modes just outside the 2/3 band and at
    the Nyquist frequencies: (j, k) = (Kx+1, 0), (Nx/2, 0), (1, Ks+1), (0, Ns/2), (Kx+1, Ks+1)
    and (Nx/2, Ns/2), with Kx = Nx // 3, Ks = Ns // 3, each a cosine of amplitude ``amp`` with
    a fixed phase.  Its projection onto the band is zero."""
    kx, ks = nx // 3, ns // 3
    m = np.arange(nx)[None, :] / nx
    n = np.arange(ns)[:, None] / ns
    out = np.zeros((ns, nx))
    for i, (j, k) in enumerate(((kx + 1, 0), (nx // 2, 0), (1, ks + 1), (0, ns // 2),
                                (kx + 1, ks + 1), (nx // 2, ns // 2))):
        out += amp * np.cos(2.0 * np.pi * (j * m + k * n) + 0.3 * (i + 1))
    return out


def make_loops(name: str, nx: int, L: float, seeds: Sequence[int], *, ns=None, ns_choices=None,
               T0=None, T_range=None, decay=(2.0, 2.0), scheme=1, dtau=0.15, meta=None,
               symmetric=False):
    us, Ts, nss = [], [], []
    for sd in seeds:
        u, T, n = spectral_loop(sd, nx, L, ns=ns, ns_choices=ns_choices, T0=T0,
                                T_range=T_range, decay=decay, symmetric=symmetric)
        us.append(u)
        Ts.append(T)
        nss.append(n)
    return Workload(name, float(L), int(nx), nss, Ts, us, scheme, float(dtau), dict(meta or {}))


# The named workloads: sizes, periods and init decay rates of the descent benchmarks.
def workload(name: str, batch: Optional[int] = None,
             seeds: Optional[Sequence[int]] = None) -> Workload:
    """The named workload; ``batch`` overrides the number of loops of the batched ones (seeds
    0..batch-1), ``seeds`` gives the loops' seeds explicitly (any workload, same recipe)."""
    def sd(default_batch: int):
        if seeds is not None:
            return list(seeds)
        return list(range(default_batch if batch is None else batch))

    if name == "single_32x32_explicit":
        return make_loops(name, 32, 22.0, sd(1) if seeds is not None else [0], ns=32, T0=40.0,
                          scheme=0, dtau=1e-4, meta={"steps": 2000})
    if name == "single_64x128_imex":
        return make_loops(name, 64, 22.0, sd(1) if seeds is not None else [0], ns=128,
                          T_range=(20.0, 80.0), scheme=1, dtau=0.15,
                          meta={"tol": 1e-10, "max_steps": 1_000_000})
    if name == "batch16_64x64":
        return make_loops(name, 64, 22.0, sd(16), ns=64, T_range=(20.0, 80.0), scheme=1,
                          dtau=0.15)
    if name == "ragged256_64xNs":
        return make_loops(name, 64, 22.0, sd(256), ns_choices=(32, 64, 128, 256),
                          T_range=(10.0, 100.0), scheme=1, dtau=0.15)
    if name == "large8_256x1024":
        return make_loops(name, 256, 100.0, sd(8), ns=1024, T0=120.0, decay=(8.0, 8.0),
                          scheme=1, dtau=0.15, meta={"switch_tol": 1e-5, "tol": 1e-10})
    if name == "paper_L39_64x64":
        # the paper's own numerical setting (Sec. 4.4): L = 39, 64 x 64 modes, dtau = 0.15,
        # T0 = 40, here on a seeded spectral loop in place of the authors' recurrence guess
        return make_loops(name, 64, 39.0, sd(1), ns=64, T0=40.0, scheme=1, dtau=0.15,
                          meta={"tol": 1e-12})
    if name == "paper_L39_xi_64x64":
        # the same setting restricted to centre-symmetric loops, as the paper's initial loops
        # and converged orbits are (Sec. 4.4); descended with the "symmetry" knob set to 1
        return make_loops(name, 64, 39.0, sd(1), ns=64, T0=40.0, scheme=1, dtau=0.15,
                          meta={"tol": 1e-12, "symmetry": 1}, symmetric=True)
    raise KeyError(name)


def orbit_guess(path: Optional[str] = None) -> Workload:
    """The stored initial loop at the paper's setting (L = 39, 64 x 64, dtau = 0.15, IMEX): a
    centre-symmetric recurrence loop of a chaotic run (Sec. 4.3), kept as band coefficients
    (``data/orbit_guess_L39.json``, written by ``data/make_orbit_guess.py``) and synthesised on
    the grid here; descended with the "symmetry" knob it converges to a periodic orbit."""
    import json
    import os
    if path is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                            "orbit_guess_L39.json")
    with open(path) as f:
        rec = json.load(f)
    nx, ns = int(rec["nx"]), int(rec["ns"])
    half = np.array(rec["c"], dtype=np.float64)            # [j-1][k][re, im], k = 0..Ks
    ch = half[..., 0] + 1j * half[..., 1]
    kx, ks = ch.shape[0], ch.shape[1] - 1
    c = np.zeros((kx + 1, 2 * ks + 1), dtype=complex)       # j = 0..Kx, k = -Ks..Ks
    c[1:, ks:] = ch
    c[1:, :ks] = -np.conj(ch[:, :0:-1])                     # c_{j,-k} = -conj(c_{j,k})
    j = np.arange(kx + 1)
    k = np.arange(-ks, ks + 1)
    ex = np.exp(2j * np.pi * np.outer(j, np.arange(nx)) / nx)
    es = np.exp(2j * np.pi * np.outer(np.arange(ns), k) / ns)
    u = 2.0 * (es @ c.T @ ex).real
    return Workload("orbit_guess_L39_xi_64x64", float(rec["L"]), nx, [ns], [float(rec["T0"])],
                    [u], 1, 0.15, {"tol": 1e-10, "symmetry": 1, "t0": rec["t0"]})


WORKLOADS = ("single_32x32_explicit", "single_64x128_imex", "batch16_64x64",
             "ragged256_64xNs", "large8_256x1024", "paper_L39_64x64", "paper_L39_xi_64x64")
