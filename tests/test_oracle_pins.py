"""Pins for the CPU oracle, each against something other than the oracle itself.

Every check here is fixed by the paper's equations or by mathematics derived by hand:
closed forms for a single Fourier mode (Eq. KS_R, Eq. cost_function, Eq. KS_L_dagger),
equilibria with zero residual (Sec. 4.1), Parseval, the adjoint identity that defines
L^dag (Eq. adjoint_definition, App. B), centred finite differences of J, the expanded flow of
Eq. KS_G_1, the shift symmetries (Sec. 3) and the centre symmetry (Sec. 4.1, Eq. KS_loop_sym), monotone decrease of J
(Eq. J_variation) and the linear decay factors of the Euler schemes (Sec. 4.2).
"""
import math

import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2007_06427_gb300.inputs import spectral_loop


def mode_field(Nx, Ns, L, j, k, a, phase=0.0):
    m = np.arange(Nx)[None, :]
    n = np.arange(Ns)[:, None]
    th = 2 * math.pi * (j * m / Nx + k * n / Ns) + phase
    return a * np.cos(th), th


def single_mode_closed_form(Nx, Ns, L, T, j, k, a):
    """Hand-derived r, J, dJ/dT, G for u = a cos(q x + w s) (see module docstring)."""
    q = 2 * math.pi * j / L
    w = 2 * math.pi * k
    u, th = mode_field(Nx, Ns, L, j, k, a)
    A = a * w / T
    B = a * (q * q - q ** 4)
    C = a * a * q / 2
    r = A * np.sin(th) + B * np.cos(th) + C * np.sin(2 * th)
    J = L * (a * a * (w * w / T ** 2 + (q * q - q ** 4) ** 2) / 2 + a ** 4 * q * q / 8)
    dJdT = -L * a * a * w * w / T ** 3
    G = ((w / T) * (A * np.cos(th) - B * np.sin(th) + 2 * C * np.cos(2 * th))
         + a * q * (A / 2 + (A / 2) * np.cos(2 * th) - (B / 2) * np.sin(2 * th)
                    + C * np.cos(th) + C * np.cos(3 * th))
         + q * q * (A * np.sin(th) + B * np.cos(th) + 4 * C * np.sin(2 * th))
         - q ** 4 * (A * np.sin(th) + B * np.cos(th) + 16 * C * np.sin(2 * th)))
    return u, r, J, dJdT, G


@pytest.mark.parametrize("Nx,Ns,L,T,j,k,a", [
    (32, 32, 22.0, 40.0, 1, 1, 0.7),
    (32, 32, 22.0, 40.0, 2, 3, 1.3),
    (32, 64, 22.0, 17.0, 3, -2, 0.4),
    (64, 32, 39.0, 55.0, 5, 1, 1.1),
    (32, 32, 22.0, 40.0, 0, 2, 0.9),     # pure temporal mode: no nonlinearity
    (32, 32, 22.0, 40.0, 3, 0, 0.9),     # steady mode: no s-derivative, dJ/dT = 0
])
def test_single_mode_closed_form(Nx, Ns, L, T, j, k, a):
    u, r_cf, J_cf, dJdT_cf, G_cf = single_mode_closed_form(Nx, Ns, L, T, j, k, a)
    # the cubic term of G lives at (3j, 3k): the closed form holds only inside the band
    assert 3 * abs(j) <= Nx // 3 and 3 * abs(k) <= Ns // 3
    res = ko.residual(u, T, L)
    np.testing.assert_allclose(res["r"], r_cf, rtol=0, atol=1e-11 * max(1, np.abs(r_cf).max()))
    assert res["J"] == pytest.approx(J_cf, rel=1e-12, abs=1e-14)
    assert res["dJdT"] == pytest.approx(dJdT_cf, rel=1e-12, abs=1e-14)
    adj = ko.adjoint_grad(u, T, L)
    np.testing.assert_allclose(adj["G"], G_cf, rtol=0, atol=1e-10 * max(1, np.abs(G_cf).max()))


def test_single_mode_truncated_cubic_term():
    """When (3j, 3k) lies outside the 2/3 band, G loses exactly the cos(3 theta) term."""
    Nx = Ns = 32
    L, T, j, k, a = 22.0, 30.0, 4, 1, 0.8
    u, r_cf, J_cf, _, G_cf = single_mode_closed_form(Nx, Ns, L, T, j, k, a)
    _, th = mode_field(Nx, Ns, L, j, k, a)
    q = 2 * math.pi * j / L
    C = a * a * q / 2
    G_trunc = G_cf - a * q * C * np.cos(3 * th)
    adj = ko.adjoint_grad(u, T, L)
    np.testing.assert_allclose(adj["G"], G_trunc, rtol=0, atol=1e-10 * np.abs(G_cf).max())
    assert adj["J"] == pytest.approx(J_cf, rel=1e-12)


@pytest.mark.parametrize("c", [0.0, 0.37, -1.5])
def test_constant_equilibria_have_zero_residual(c):
    """u = const is an equilibrium of KS (Sec. 4.1): r = 0, G = 0, J = dJ/dT = 0."""
    u = np.full((16, 32), c)
    res = ko.residual(u, 33.0, 22.0)
    adj = ko.adjoint_grad(u, 33.0, 22.0)
    assert np.abs(res["r"]).max() < 1e-13
    assert np.abs(adj["G"]).max() < 1e-11   # rounding noise amplified by q^4 multipliers
    assert res["J"] < 1e-24 and abs(res["dJdT"]) < 1e-24


def test_parseval():
    """J from the grid (oracle) equals L * sum |r_hat|^2 over the full spectrum."""
    u, T, _ = spectral_loop(3, 32, 22.0, ns=64, T0=35.0)
    res = ko.residual(u, T, 22.0)
    J_spec = 22.0 * float(np.sum(np.abs(res["rh"]) ** 2))
    assert res["J"] == pytest.approx(J_spec, rel=1e-13)


def _band_random(rng, Nx, Ns, L, shrink=1):
    """Random real band-limited field with modes |j| <= Kx/shrink, |k| <= Ks/shrink."""
    g = ko.grid(Nx, Ns, L)
    f = rng.standard_normal((Ns, Nx))
    fh = g.to_spectral(f)
    kx, ks = (Nx // 3) // shrink, (Ns // 3) // shrink
    keep = (np.abs(g.k)[:, None] <= ks) & (np.abs(g.j)[None, :] <= kx)
    return g.real_grid(np.where(keep, fh, 0)) * math.sqrt(Nx * Ns) / 4


@pytest.mark.parametrize("Nx,Ns", [(16, 16), (32, 16), (16, 32)])
def test_adjoint_identity(Nx, Ns):
    """<L(u; [v; v2]), [w; 0]> = <[v; v2], L^dag(u; [w; 0])> (Eq. adjoint_definition)."""
    rng = np.random.default_rng(7)
    L, T = 22.0, 41.0
    u = _band_random(rng, Nx, Ns, L)
    v = _band_random(rng, Nx, Ns, L)
    w = _band_random(rng, Nx, Ns, L)
    v2 = 0.83
    lhs_field = ko.directional_derivative(u, T, v, v2, L)
    lhs = L * np.mean(lhs_field * w)
    adj_field, adj_scalar = ko.adjoint_operator(u, T, w, L)
    rhs = L * np.mean(v * adj_field) + v2 * adj_scalar
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("Nx,Ns", [(8, 8), (16, 16)])
def test_gradient_matches_finite_differences(Nx, Ns):
    """dJ along a direction v equals (2L/(Nx Ns)) sum_grid G v, and dJ/dT = 2 L^dag_2.

    Centred differences with h = 1e-6; the exact gradient of the discrete J is what the
    dealiased two-stage evaluation returns.
    """
    rng = np.random.default_rng(11)
    L, T, h = 22.0, 37.0, 1e-6
    u = _band_random(rng, Nx, Ns, L)
    adj = ko.adjoint_grad(u, T, L)
    for _ in range(3):
        v = rng.standard_normal((Ns, Nx))          # any grid direction: J sees P v
        Jp = ko.residual(u + h * v, T, L)["J"]
        Jm = ko.residual(u - h * v, T, L)["J"]
        fd = (Jp - Jm) / (2 * h)
        an = 2 * L / (Nx * Ns) * float(np.sum(adj["G"] * v))
        assert fd == pytest.approx(an, rel=2e-7, abs=1e-9)
    fdT = (ko.residual(u, T + h, L)["J"] - ko.residual(u, T - h, L)["J"]) / (2 * h)
    assert fdT == pytest.approx(adj["dJdT"], rel=2e-7, abs=1e-9)
    # per grid value as well (J is defined on P u)
    for idx in [(0, 0), (Ns // 2, 3), (Ns - 1, Nx - 1)]:
        e = np.zeros((Ns, Nx))
        e[idx] = 1.0
        fd = (ko.residual(u + h * e, T, L)["J"] - ko.residual(u - h * e, T, L)["J"]) / (2 * h)
        an = 2 * L / (Nx * Ns) * adj["G"][idx]
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("Nx,Ns,L,T", [(32, 32, 22.0, 40.0), (64, 32, 39.0, 60.0)])
def test_expanded_flow_matches_two_stage(Nx, Ns, L, T):
    """-L^dag_1 r (two stages) equals G_1,L + G_1,NL of Eq. KS_G_1 on loops whose band is
    narrow enough (|j| <= Nx/8, |k| <= Ns/8) that the cubic products do not alias."""
    rng = np.random.default_rng(5)
    g = ko.grid(Nx, Ns, L)
    f = rng.standard_normal((Ns, Nx))
    fh = g.to_spectral(f)
    keep = (np.abs(g.k)[:, None] <= Ns // 8) & (np.abs(g.j)[None, :] <= Nx // 8)
    u = g.real_grid(np.where(keep, fh, 0)) * 6
    two_stage = -ko.adjoint_grad(u, T, L)["G"]
    expanded = ko.flow_expanded(u, T, L)
    scale = np.abs(two_stage).max()
    np.testing.assert_allclose(expanded, two_stage, rtol=0, atol=1e-11 * scale)


def test_shift_equivariance():
    """r and G commute with grid shifts in x and s (Sec. 3: J is invariant to s-phase)."""
    u, T, _ = spectral_loop(2, 32, 22.0, ns=32, T0=40.0)
    a = ko.adjoint_grad(u, T, 22.0)
    for ax, sh in [(1, 5), (0, 7)]:
        b = ko.adjoint_grad(np.roll(u, sh, axis=ax), T, 22.0)
        np.testing.assert_allclose(b["G"], np.roll(a["G"], sh, axis=ax), atol=1e-10)
        assert b["J"] == pytest.approx(a["J"], rel=1e-12)
        assert b["dJdT"] == pytest.approx(a["dJdT"], rel=1e-10, abs=1e-12)


def _xi(u):
    """Xi of Eq. KS_loop_sym on the grid: u(x, s) -> -u(-x, s)."""
    return -np.roll(u[:, ::-1], 1, axis=1)


def test_center_symmetry_preserved():
    """A Xi-invariant loop stays Xi-invariant under the tau-flow (Eq. KS_loop_sym)."""
    u0, T, _ = spectral_loop(4, 32, 22.0, ns=32, T0=40.0)
    u = 0.5 * (u0 + _xi(u0))
    assert np.abs(u - _xi(u)).max() < 1e-14
    out = ko.descend(u, T, 22.0, 0.15, ko.IMEX, 5)
    v = out["u"]
    assert np.abs(v - _xi(v)).max() < 1e-12 * np.abs(v).max()
    G = ko.adjoint_grad(u, T, 22.0)["G"]
    assert np.abs(G - _xi(G)).max() < 1e-11 * np.abs(G).max()


def test_xi_projection_matches_grid_reflection():
    """The spectral Xi projection equals the transform of (u(x, s) - u(-x, s)) / 2 formed on
    the grid (Eq. KS_loop_sym), for an arbitrary field (all modes, Nyquist included)."""
    rng = np.random.default_rng(21)
    for Nx, Ns in [(8, 8), (16, 32), (32, 16)]:
        g = ko.grid(Nx, Ns, 22.0)
        u = rng.standard_normal((Ns, Nx))
        spec = g.xi_project(g.to_spectral(u))
        grid_side = g.to_spectral(0.5 * (u + _xi(u)))
        np.testing.assert_allclose(spec, grid_side, rtol=0, atol=1e-15)


def test_xi_projection_closed_forms():
    """sin(q x) f(s) is Xi-invariant, cos(q x) f(s) is projected out; the projector is
    idempotent and self-adjoint (an orthogonal projection)."""
    Nx, Ns, L = 32, 32, 22.0
    g = ko.grid(Nx, Ns, L)
    x = L * np.arange(Nx)[None, :] / Nx
    s = np.arange(Ns)[:, None] / Ns
    f = np.cos(2 * math.pi * s) + 0.3 * np.sin(4 * math.pi * s + 0.2)
    odd = np.sin(2 * math.pi * 3 * x / L) * f
    even = np.cos(2 * math.pi * 2 * x / L) * f + 0.7
    np.testing.assert_allclose(ko.band_state(odd, L, xi=True), ko.band_state(odd, L), atol=1e-15)
    assert np.abs(ko.band_state(even, L, xi=True)).max() < 1e-15
    np.testing.assert_allclose(ko.band_state(odd + even, L, xi=True), ko.band_state(odd, L),
                               atol=1e-15)
    rng = np.random.default_rng(3)
    a = g.to_spectral(rng.standard_normal((Ns, Nx)))
    b = g.to_spectral(rng.standard_normal((Ns, Nx)))
    np.testing.assert_allclose(g.xi_project(g.xi_project(a)), g.xi_project(a), atol=1e-16)
    lhs = np.vdot(g.xi_project(a), b)
    rhs = np.vdot(a, g.xi_project(b))
    assert abs(lhs - rhs) < 1e-15


def test_xi_descent_equals_plain_descent_on_invariant_loop():
    """On a Xi-invariant loop the projected descent follows the unprojected one (the flow
    preserves the symmetry, Sec. 4.1): they differ by rounding only."""
    u, T, _ = spectral_loop(4, 32, 22.0, ns=32, T0=40.0, symmetric=True)
    a = ko.descend(u, T, 22.0, 0.15, ko.IMEX, 8)
    b = ko.descend(u, T, 22.0, 0.15, ko.IMEX, 8, xi=True)
    assert np.abs(a["u"] - b["u"]).max() < 1e-13 * np.abs(a["u"]).max()
    assert b["T"] == pytest.approx(a["T"], rel=1e-14)
    assert np.abs(b["u"] - _xi(b["u"])).max() < 1e-14 * np.abs(b["u"]).max()


@pytest.mark.parametrize("Nx,Ns", [(8, 8), (16, 16)])
def test_xi_gradient_matches_finite_differences(Nx, Ns):
    """With xi, J(u) := J(P_Xi P u) and the returned G is its gradient: centred differences
    along arbitrary (not invariant) directions from a non-invariant u match
    (2L/(Nx Ns)) sum_grid G v."""
    rng = np.random.default_rng(17)
    L, T, h = 22.0, 33.0, 1e-6
    u = _band_random(rng, Nx, Ns, L)
    adj = ko.adjoint_grad(u, T, L, xi=True)
    assert np.abs(adj["G"] - _xi(adj["G"])).max() < 1e-13 * np.abs(adj["G"]).max()
    for _ in range(3):
        v = rng.standard_normal((Ns, Nx))
        fd = (ko.residual(u + h * v, T, L, xi=True)["J"]
              - ko.residual(u - h * v, T, L, xi=True)["J"]) / (2 * h)
        an = 2 * L / (Nx * Ns) * float(np.sum(adj["G"] * v))
        assert fd == pytest.approx(an, rel=2e-7, abs=1e-9)
    fdT = (ko.residual(u, T + h, L, xi=True)["J"] - ko.residual(u, T - h, L, xi=True)["J"]) / (2 * h)
    assert fdT == pytest.approx(adj["dJdT"], rel=2e-7, abs=1e-9)


def test_monotone_decrease_explicit():
    """J decreases at every one of 2000 explicit steps (Eq. J_variation), 32 x 32, L = 22."""
    u, T, _ = spectral_loop(0, 32, 22.0, ns=32, T0=40.0)
    out = ko.descend(u, T, 22.0, 1e-4, ko.EXPLICIT, 2000, record=True)
    h = out["hist"]
    assert len(h) == 2001
    assert np.all(np.diff(h) < 0)
    assert h[-1] < 0.5 * h[0]


def test_monotone_decrease_imex():
    """With the paper's step (dtau = 0.15) the IMEX descent also decreases J."""
    u, T, _ = spectral_loop(1, 32, 22.0, ns=32, T0=40.0)
    out = ko.descend(u, T, 22.0, 0.15, ko.IMEX, 200, record=True)
    assert np.all(np.diff(out["hist"]) < 0)


@pytest.mark.parametrize("scheme", [ko.EXPLICIT, ko.IMEX])
def test_linear_regime_decay_factor(scheme):
    """For amplitude -> 0 each band mode is multiplied per step by 1 + dtau*Lambda_jk
    (explicit) or 1/(1 - dtau*Lambda_jk) (IMEX), Lambda_jk of Sec. 4.2 written out here."""
    Nx = Ns = 32
    L, T, eps = 22.0, 40.0, 1e-9
    dtau = 1e-4 if scheme == ko.EXPLICIT else 0.15
    for (j, k) in [(1, 0), (2, 1), (5, -3), (0, 4)]:
        u, _ = mode_field(Nx, Ns, L, j, k, eps)
        out = ko.descend(u, T, L, dtau, scheme, 1)
        q = 2 * math.pi * j / L
        w = 2 * math.pi * k
        lam = -(w / T) ** 2 - q ** 8 + 2 * q ** 6 - q ** 4
        fac = 1 + dtau * lam if scheme == ko.EXPLICIT else 1 / (1 - dtau * lam)
        np.testing.assert_allclose(out["u"], fac * u, rtol=0, atol=1e-6 * eps)
        assert abs(out["T"] - T) < 1e-12


def test_descend_stops_at_tolerance():
    u = np.zeros((16, 16))
    out = ko.descend(u, 30.0, 22.0, 0.15, ko.IMEX, 100, tol=1e-10)
    assert out["steps"] == 0 and out["sqrtJ"] == 0.0


# ---------------------------------------------------------------------------------------
# Extrapolation along the trajectory (App. C)
# ---------------------------------------------------------------------------------------

def test_extrapolation_is_exact_on_one_decaying_eigendirection():
    """A tiny single Fourier mode is in the linear regime: every IMEX step multiplies it by
    1/(1 - dtau Lambda_jk), so sqrt(J) falls geometrically along one eigendirection and the
    geometric extrapolation of App. C lands on the fixed point u = 0 up to the O(a^2) harmonic
    and rounding.  A wrong coefficient, sign or anchor would leave a finite fraction."""
    Nx = Ns = 16
    L, T, a = 22.0, 40.0, 1e-9
    j, k = 2, 1
    u, _ = mode_field(Nx, Ns, L, j, k, a)
    q, w = 2 * math.pi * j / L, 2 * math.pi * k
    lam = -(w / T) ** 2 - q ** 8 + 2 * q ** 6 - q ** 4
    fac = 1.0 / (1.0 - 0.15 * lam)
    assert fac ** 100 < 0.5                      # one chunk halves sqrt(J)
    # anchor at step 100, extrapolation at step 200 (nsteps = 200: no step after it)
    out = ko.descend_extrapolated(u, T, L, 0.15, ko.IMEX, 200, 0.0, 100, start=1.0)
    assert out["steps"] == 200 and out["extrapolations"] == 1 and out["rejected"] == 0
    plain = ko.descend(u, T, L, 0.15, ko.IMEX, 200)
    sq_b = plain["sqrtJ"]
    np.testing.assert_allclose(plain["u"], fac ** 200 * u, rtol=0, atol=1e-6 * a * fac ** 200)
    assert out["sqrtJ"] < 1e-6 * sq_b
    assert np.abs(out["u"]).max() < 1e-6 * a * fac ** 200
    assert abs(out["T"] - T) < 1e-12


def test_extrapolation_off_is_the_plain_descent():
    """With no observation at or below the start threshold the chunked descent is the plain
    descent, step for step and bit for bit."""
    u0, T0, _ = spectral_loop(3, 16, 22.0, ns=16, T_range=(30.0, 50.0))
    u0 = 1e-2 * u0
    plain = ko.descend(u0, T0, 22.0, 0.15, ko.IMEX, 230)
    ext = ko.descend_extrapolated(u0, T0, 22.0, 0.15, ko.IMEX, 230, 0.0, 70, start=0.0)
    assert ext["steps"] == plain["steps"] == 230
    assert ext["extrapolations"] == 0 and ext["rejected"] == 0
    assert ext["T"] == plain["T"]
    np.testing.assert_array_equal(ext["u"], plain["u"])


def test_extrapolation_never_raises_sqrtJ_and_saves_steps():
    """An extrapolated state is kept only if it lowers sqrt(J); on a small loop in its
    exponential tail the accelerated descent reaches 1e-8 in fewer steps than the plain one
    (App. C reports more than half the steps saved on its example)."""
    u0, T0, _ = spectral_loop(3, 16, 22.0, ns=16, T_range=(30.0, 50.0))
    u0 = 1e-2 * u0
    ext = ko.descend_extrapolated(u0, T0, 22.0, 0.15, ko.IMEX, 6000, 1e-8, 100)
    assert ext["sqrtJ"] < 1e-8 and ext["extrapolations"] >= 2
    plain = ko.descend(u0, T0, 22.0, 0.15, ko.IMEX, ext["steps"], tol=1e-8)
    assert plain["sqrtJ"] > 1e-6              # the plain descent is still far from 1e-8 there
