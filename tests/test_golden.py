"""Stored values in tests/golden: the paper's printed settings (each with its passage) and the
oracle's outputs on single-mode loops (written by tests/golden/make_golden.py, which calls only
the oracle).  The oracle must still reproduce them, and they must equal the hand-derived closed
forms of Eq. KS_R, Eq. cost_function and Eq. KS_L_dagger for u = a cos(q x + omega s)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2007_06427_gb300.inputs import workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_oracle_reproduces_its_stored_single_mode_values():
    for c in load("oracle_single_mode.json")["cases"]:
        Nx, Ns, L, T, j, k, a = (c[key] for key in ("Nx", "Ns", "L", "T", "j", "k", "a"))
        m = np.arange(Nx)[None, :]
        n = np.arange(Ns)[:, None]
        u = a * np.cos(2 * math.pi * (j * m / Nx + k * n / Ns))
        res = ko.adjoint_grad(u, T, L)
        r = ko.residual(u, T, L)["r"]
        assert res["J"] == pytest.approx(c["J"], rel=1e-13, abs=1e-300)
        assert res["dJdT"] == pytest.approx(c["dJdT"], rel=1e-12, abs=1e-15)
        for (pn, pm, v) in c["r"]:
            assert r[pn % Ns, pm % Nx] == pytest.approx(v, rel=1e-12, abs=1e-14)
        for (pn, pm, v) in c["G"]:
            assert res["G"][pn % Ns, pm % Nx] == pytest.approx(v, rel=1e-12, abs=1e-12)


def test_stored_values_equal_closed_forms():
    """J = L [a^2 (w^2/T^2 + (q^2 - q^4)^2) / 2 + a^4 q^2 / 8], dJ/dT = -L a^2 w^2 / T^3, and
    r = (a w / T) sin th + a (q^2 - q^4) cos th + (a^2 q / 2) sin 2 th at the stored points."""
    for c in load("oracle_single_mode.json")["cases"]:
        Nx, Ns, L, T, j, k, a = (c[key] for key in ("Nx", "Ns", "L", "T", "j", "k", "a"))
        q = 2 * math.pi * j / L
        w = 2 * math.pi * k
        J = L * (a * a * (w * w / T ** 2 + (q * q - q ** 4) ** 2) / 2 + a ** 4 * q * q / 8)
        assert c["J"] == pytest.approx(J, rel=1e-12)
        assert c["dJdT"] == pytest.approx(-L * a * a * w * w / T ** 3, rel=1e-10, abs=1e-15)
        for (pn, pm, v) in c["r"]:
            th = 2 * math.pi * (j * (pm % Nx) / Nx + k * (pn % Ns) / Ns)
            rv = (a * w / T) * math.sin(th) + a * (q * q - q ** 4) * math.cos(th) \
                + (a * a * q / 2) * math.sin(2 * th)
            assert v == pytest.approx(rv, rel=1e-11, abs=1e-13)


def test_paper_setting_workloads_match_the_printed_parameters():
    ps = load("paper_setting.json")
    for name in ("paper_L39_64x64", "paper_L39_xi_64x64"):
        w = workload(name)
        assert w.L == ps["L"]["value"]
        assert [w.nx, w.ns[0]] == ps["modes"]["value"]
        assert w.dtau == ps["dtau"]["value"]
        assert w.T0[0] == ps["T0"]["value"]
        assert w.meta["tol"] == ps["tol"]["value"]
        assert w.scheme == 1                                   # IMEX Euler (Sec. 4.2)
    # the printed convergence time corresponds to ~1e7 steps of the printed step
    assert ps["tau_converged"]["value"] / ps["dtau"]["value"] == pytest.approx(1e7, rel=0.01)


def test_trivial_solution_unstable_above_2pi():
    """u = const is linearly unstable exactly when the first mode q_1 = 2 pi / L has
    q^2 - q^4 > 0, i.e. L > 2 pi (Sec. 4): the oracle's linear residual symbol agrees."""
    Lc = load("paper_setting.json")["trivial_unstable_above"]["value"]
    for L, unstable in ((0.99 * Lc, False), (1.01 * Lc, True), (39.0, True)):
        g = ko.grid(16, 8, L)
        j1 = g.Nx // 2 + 1                       # signed mode j = 1 on axis 1
        k0 = g.Ns // 2                           # k = 0
        uh = np.zeros((g.Ns, g.Nx), dtype=complex)
        uh[k0, j1] = 1e-8
        uh[k0, g.Nx // 2 - 1] = 1e-8             # its conjugate, real field
        rh, _, _ = ko.residual_hat(uh, 50.0, g)
        # r = -(u_xx + u_xxxx) at linear order: r_hat = (q^2 - q^4) u_hat; growth rate of the
        # KSE linear part is q^2 - q^4 = r_hat / u_hat
        growth = (rh[k0, j1] / uh[k0, j1]).real
        assert (growth > 0) == unstable
