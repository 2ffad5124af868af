"""Initial loops from recurrences of a chaotic KS run (Sec. 4.3): the time stepper is pinned
by the exact linear evolution of a single mode and the conserved mean; extracted loops are
band limited and lie far closer to solutions than random loops of the same size."""
import math

import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2007_06427_gb300.guesses import chaotic_run, ks_dns, norm_series, recurrence_loops
from paper_2007_06427_gb300.inputs import spectral_loop


@pytest.mark.parametrize("j", [1, 2, 3])
def test_dns_linear_mode_is_exact(j):
    """ETDRK4 integrates the linear part exactly: a mode of amplitude 1e-12 (nonlinear part
    ~1e-24) grows or decays by exp((q^2 - q^4) t)."""
    L, nx = 22.0, 32
    x = L * np.arange(nx) / nx
    q = 2 * math.pi * j / L
    _, us = ks_dns(L, nx, 0.25, 40, 1e-12 * np.cos(q * x), save_every=40)
    exact = 1e-12 * math.exp((q * q - q ** 4) * 10.0) * np.cos(q * x)
    np.testing.assert_allclose(us[-1], exact, rtol=0, atol=1e-9 * np.abs(exact).max())


def test_dns_conserves_mean_and_stays_bounded():
    ts, us = chaotic_run(22.0, 32, 400.0, seed=1)
    means = us.mean(axis=1)
    assert np.abs(means - means[0]).max() < 1e-13
    nrm = norm_series(us, 22.0)
    assert np.isfinite(nrm).all() and 1.0 < nrm[-200:].mean() < 30.0


def test_recurrence_loops_are_band_limited_near_solutions():
    L, nx, ns = 22.0, 32, 32
    ts, us = chaotic_run(L, nx, 2000.0, seed=0)
    loops = recurrence_loops(ts, us, L, ns, T_range=(10.0, 80.0), tol=0.005, t_min=200.0,
                             max_loops=3)
    assert len(loops) >= 1
    g = ko.grid(nx, ns, L)
    rnd, _, _ = spectral_loop(0, nx, L, ns=ns, T0=40.0)
    for lp in loops:
        assert 10.0 <= lp.T <= 80.0 and lp.mismatch < 0.005
        spec = g.to_spectral(lp.u)
        outside = np.abs(np.where(g.mask, 0, spec)).max()
        assert outside < 1e-12 * np.abs(spec).max()
        e = L * np.mean(lp.u ** 2)
        J = ko.residual(lp.u, lp.T, L)["J"]
        r = rnd * math.sqrt(np.mean(lp.u ** 2))
        J_rnd = ko.residual(r, lp.T, L)["J"]
        assert J / e < 0.2 and J < 0.1 * J_rnd


def _reflect(u):
    """u(-x) on the grid x_m = m L / Nx (last axis)."""
    return np.roll(u[..., ::-1], 1, axis=-1)


def test_symmetric_run_and_loops_stay_centre_symmetric():
    """In the centre-symmetric subspace (Sec. 4.4) the run stays odd in x and chaotic, and the
    extracted loops are odd in x as well (L = 39, the paper's domain)."""
    L, nx, ns = 39.0, 64, 64
    ts, us = chaotic_run(L, nx, 1500.0, seed=2, symmetric=True)
    assert np.abs(us + _reflect(us)).max() < 1e-13 * np.abs(us).max()
    nrm = norm_series(us, L)
    tail = nrm[-400:]
    assert np.isfinite(nrm).all() and tail.mean() > 1.0 and np.ptp(tail) > 0.05 * tail.mean()
    loops = recurrence_loops(ts, us, L, ns, T_range=(10.0, 120.0), tol=0.01, t_min=200.0,
                             max_loops=2)
    assert len(loops) >= 1
    for lp in loops:
        assert np.abs(lp.u + _reflect(lp.u)).max() < 1e-12 * np.abs(lp.u).max()
        # the oracle's Xi projection leaves it unchanged
        np.testing.assert_allclose(ko.band_state(lp.u, L, xi=True), ko.band_state(lp.u, L),
                                   rtol=0, atol=1e-13 * np.abs(lp.u).max())


def test_orbit_classification_closed_forms():
    """u = 0 is trivial, u = a sin(q x) is steady, u = a sin(q x + 2 pi s) has
    ||u_s|| / ||u|| = 2 pi (omega = 2 pi for the first temporal mode)."""
    from paper_2007_06427_gb300.orbits import classify
    L, nx, ns = 39.0, 32, 32
    x = L * np.arange(nx)[None, :] / nx
    s = np.arange(ns)[:, None] / ns
    q = 2 * math.pi * 2 / L
    assert classify(np.zeros((ns, nx)), L)[0] == "trivial"
    kind, norm, ratio = classify(0.7 * np.sin(q * x) + 0 * s, L)
    assert kind == "steady" and ratio < 1e-14 and norm == pytest.approx(0.7 * math.sqrt(L / 2))
    kind, norm, ratio = classify(0.7 * np.sin(q * x + 2 * math.pi * s), L)
    assert kind == "periodic" and ratio == pytest.approx(2 * math.pi, rel=1e-12)


def test_dns_is_fourth_order_on_a_chaotic_state():
    """ETDRK4 is a fourth-order scheme: from a state on the chaotic attractor (L = 22, Nx = 64),
    halving dt divides the error at t = 1 by a factor that approaches 2^4 = 16 (a scheme of order
    three or two would approach 8 or 4).  Measured against a run with dt = 1/2048."""
    L, nx = 22.0, 64
    _, us = chaotic_run(L, nx, 300.0, seed=1)
    u0 = us[-1]

    def run(dt):
        n = int(round(1.0 / dt))
        return ks_dns(L, nx, dt, n, u0, save_every=n)[1][-1]

    ref = run(1.0 / 2048)
    errs = [np.abs(run(dt) - ref).max() for dt in (1 / 64, 1 / 128, 1 / 256)]
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert ratios[1] > ratios[0] > 11.0, ratios
    assert math.log2(ratios[1]) > 3.7, ratios


def test_dns_time_derivative_is_the_ks_right_hand_side():
    """The DNS advances u_t = -u u_x - u_xx - u_xxxx: its centred difference in time on a chaotic
    state equals the oracle's right-hand side N(P u) of the same snapshot (the oracle's residual
    of a loop constant in s, where -(1/T) u_s vanishes).  Pins the sign and the factor of the
    nonlinear term and its dealiasing independently of the exactness of the linear part."""
    L, nx, h = 22.0, 64, 1e-4
    _, us = chaotic_run(L, nx, 300.0, seed=1)
    u0 = us[-1]
    _, fine = ks_dns(L, nx, h / 8, 16, u0, save_every=8)        # u(0), u(h), u(2h)
    dudt = (fine[2] - fine[0]) / (2 * h)
    loop = np.repeat(fine[1][None, :], 8, axis=0)
    N = ko.residual(loop, 40.0, L)["r"][0]
    # the centred difference is second order in h: ~1.5e-7 at h = 1e-4 (1.1e-5 at h = 1e-3)
    assert np.abs(dudt - N).max() < 1e-6 * np.abs(N).max()
