"""Write ``orbit_guess_L39.json``: one initial loop at the paper's setting (L = 39, 64 x 64,
centre-symmetric) taken from a close recurrence of a chaotic KS run (Sec. 4.3), stored as its
band coefficients so that every machine starts from the same loop.

A chaotic run is not reproducible bit for bit on other hardware or with other transforms
(different rounding grows exponentially along the trajectory), which is why the loop is stored
rather than recomputed.  The run and the extraction are those of ``paper_2007_06427_gb300.guesses``
(on the GPU) with the arguments below; the recurrence is chosen by its start time in the run.
Needs a CUDA device.

    python -m paper_2007_06427_gb300.data.make_orbit_guess [t0]
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "orbit_guess_L39.json")
L, NX, NS = 39.0, 64, 64
RUN = {"t_end": 6000.0, "seed": 2, "symmetric": True}
EXTRACT = {"T_range": [20.0, 32.0], "tol": 0.01, "t_min": 200.0, "max_loops": 8}


def main(t0: float = 1515.0) -> str:
    from paper_2007_06427_gb300.guesses import chaotic_run, recurrence_loops
    run = chaotic_run(L, NX, RUN["t_end"], seed=RUN["seed"], symmetric=RUN["symmetric"])
    gs = recurrence_loops(run, L, NS, T_range=tuple(EXTRACT["T_range"]), tol=EXTRACT["tol"],
                          t_min=EXTRACT["t_min"], max_loops=EXTRACT["max_loops"])
    g = min(gs, key=lambda g: abs(g.t0 - t0))
    # c_jk of u(x_m, s_n) = sum_{j, k} c_jk exp(2 pi i (m j / Nx + n k / Ns)), j = 1..Kx, k = 0..Ks;
    # the loop is odd in x, so c_{j,-k} = -conj(c_jk), and the j = 0 column is zero
    kx, ks = NX // 3, NS // 3
    c = np.fft.fft2(g.u) / (NX * NS)                 # axis 0: k (s), axis 1: j (x)
    half = np.stack([c[np.arange(ks + 1), j] for j in range(1, kx + 1)])   # [j-1][k]
    rec = {"L": L, "nx": NX, "ns": NS, "T0": g.T, "t0": g.t0, "mismatch": g.mismatch,
           "run": RUN, "extract": EXTRACT,
           "layout": "c[j-1][k] for j = 1..Nx//3, k = 0..Ns//3 as [re, im]; c[j][-k] = -conj(c[j][k])",
           "c": [[[float(v.real), float(v.imag)] for v in row] for row in half]}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=0)
    return OUT


if __name__ == "__main__":
    print(main(*(float(a) for a in sys.argv[1:])))
