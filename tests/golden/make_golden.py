"""Writes oracle_single_mode.json: the oracle's J and dJ/dT (and r, G at a few grid points) for
single-Fourier-mode loops u = a cos(q x + omega s).  Calls only the oracle; run from the
repository root:  python tests/golden/make_golden.py"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import ks_oracle as ko  # noqa: E402

CASES = [  # Nx, Ns, L, T, j, k, a
    (32, 32, 22.0, 40.0, 1, 1, 0.7),
    (32, 32, 22.0, 40.0, 2, 3, 1.3),
    (32, 64, 22.0, 17.0, 3, -2, 0.4),
    (64, 64, 39.0, 40.0, 5, 1, 1.1),
    (64, 64, 39.0, 40.0, 0, 2, 0.9),
    (64, 64, 39.0, 40.0, 3, 0, 0.9),
]
POINTS = [(0, 0), (3, 5), (17, 11)]   # (n, m) grid samples of r and G


def main():
    rows = []
    for Nx, Ns, L, T, j, k, a in CASES:
        m = np.arange(Nx)[None, :]
        n = np.arange(Ns)[:, None]
        u = a * np.cos(2 * math.pi * (j * m / Nx + k * n / Ns))
        res = ko.adjoint_grad(u, T, L)
        r = ko.residual(u, T, L)["r"]
        rows.append({"Nx": Nx, "Ns": Ns, "L": L, "T": T, "j": j, "k": k, "a": a,
                     "J": res["J"], "dJdT": res["dJdT"],
                     "r": [[p[0], p[1], float(r[p[0] % Ns, p[1] % Nx])] for p in POINTS],
                     "G": [[p[0], p[1], float(res["G"][p[0] % Ns, p[1] % Nx])] for p in POINTS]})
    out = {"note": "written by tests/golden/make_golden.py from oracle/ks_oracle.py; "
                   "u = a cos(2 pi (j m / Nx + k n / Ns)) on the grid (n, m)",
           "cases": rows}
    with open(os.path.join(HERE, "oracle_single_mode.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
