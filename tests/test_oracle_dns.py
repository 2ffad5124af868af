"""Pins of the oracle's KSE integrator (``oracle.ks_oracle.dns``), the reference for the initial
guesses of Sec. 4.3, against what the mathematics fixes:

* the phi-functions against high-precision values of their closed forms (mpmath) and their
  values at 0 (1/k!);
* a constant field is a solution and stays exactly constant; the spatial mean is conserved;
* a field of amplitude 1e-12 grows or decays by e^{(q^2 - q^4) t} (the linear symbol's sign and
  powers, with the product negligible);
* fourth-order convergence under step halving, and agreement with classical RK4 at a step far
  inside RK4's stability limit (an independent integrator of the same semi-discrete system);
* the centre-symmetric subspace u(-x) = -u(x) kept exactly.
The GPU integrator of the package is checked against it in ``test_gpu_dns.py``.
"""
import math

import numpy as np
import pytest

from oracle import ks_oracle as ko


def field(L, nx, amp=(0.5, 0.3, 0.1)):
    x = L * np.arange(nx) / nx
    return (amp[0] * np.cos(2 * np.pi * x / L) + amp[1] * np.sin(4 * np.pi * x / L)
            + amp[2] * np.cos(6 * np.pi * x / L + 0.3))


def test_phi_functions_match_closed_forms_at_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    zs = np.array([-1700.0, -50.0, -3.0, -1.0, -0.999, -1e-3, 0.0, 1e-3, 0.5, 0.999, 1.0, 2.0])
    p1, p2, p3 = ko.etd_phi(zs)
    for z, a, b, c in zip(zs, p1, p2, p3):
        if z == 0.0:
            ref = (1.0, 0.5, 1.0 / 6.0)
        else:
            Z = mp.mpf(z)
            e = mp.exp(Z)
            ref = (float((e - 1) / Z), float((e - 1 - Z) / Z ** 2), float((e - 1 - Z - Z ** 2 / 2) / Z ** 3))
        for got, want in zip((a, b, c), ref):
            assert abs(got - want) <= 2e-15 * abs(want), (z, got, want)


def test_constant_field_stays_constant_and_mean_is_conserved():
    L, nx = 22.0, 32
    _, us = ko.dns(L, nx, 0.25, 20, np.full(nx, 0.7), save_every=20)
    assert np.abs(us[-1] - 0.7).max() < 1e-15
    u0 = field(L, nx) + 0.2
    _, us = ko.dns(L, nx, 0.25, 200, u0, save_every=50)
    assert np.abs(us.mean(axis=1) - u0.mean()).max() < 1e-13


@pytest.mark.parametrize("j", [1, 3])
def test_small_amplitude_mode_follows_the_linear_symbol(j):
    """L = 22: mode 1 (q^2 - q^4 > 0) grows, mode 3 decays; the product term is ~1e-24."""
    L, nx, t = 22.0, 32, 2.0
    q = 2 * np.pi * j / L
    x = L * np.arange(nx) / nx
    eps = 1e-12
    _, us = ko.dns(L, nx, 0.01, int(round(t / 0.01)), eps * np.cos(q * x), save_every=200)
    want = eps * math.exp((q ** 2 - q ** 4) * t) * np.cos(q * x)
    assert np.abs(us[-1] - want).max() <= 1e-9 * np.abs(want).max()


def test_fourth_order_and_agreement_with_rk4():
    L, nx = 22.0, 32
    u0 = field(L, nx)
    ref = ko.dns_rk4(L, nx, 2e-4, 5000, u0)        # t = 1, |dt lambda| < 0.02
    err = []
    for dt in (0.05, 0.025):
        n = int(round(1.0 / dt))
        _, us = ko.dns(L, nx, dt, n, u0, save_every=n)
        err.append(np.abs(us[-1] - ref).max() / np.abs(ref).max())
    assert 12.0 < err[0] / err[1] < 20.0, err        # 2^4 = 16
    assert err[1] < 1e-9, err


def test_centre_symmetric_subspace_is_kept_exactly():
    L, nx = 22.0, 32
    x = L * np.arange(nx) / nx
    u0 = 0.8 * np.sin(2 * np.pi * x / L) - 0.4 * np.sin(6 * np.pi * x / L)
    _, us = ko.dns(L, nx, 0.25, 400, u0, save_every=100, symmetric=True)
    mirror = us[:, (-np.arange(nx)) % nx]                # u(-x) on the grid
    assert np.abs(us + mirror).max() < 1e-13 * np.abs(us).max()
    assert np.abs(us[-1]).max() > 0.1                    # a nontrivial state

