"""The seeded synthetic inputs: every named workload has the shape, periods, scheme and step of
its configuration, and every loop follows the recipe (zero spatial mean, grid rms 1, band
limited to |j| <= Nx/3, |k| <= Ns/3, reproducible from its seed)."""
import numpy as np
import pytest

from paper_2007_06427_gb300 import inputs
from paper_2007_06427_gb300.inputs import spectral_loop

EXPECTED = {
    # name: (loops, L, Nx, Ns set, T0 range (lo, hi) or fixed, scheme, dtau)
    "single_32x32_explicit": (1, 22.0, 32, {32}, (40.0, 40.0), 0, 1e-4),
    "single_64x128_imex": (1, 22.0, 64, {128}, (20.0, 80.0), 1, 0.15),
    "batch16_64x64": (16, 22.0, 64, {64}, (20.0, 80.0), 1, 0.15),
    "ragged256_64xNs": (256, 22.0, 64, {32, 64, 128, 256}, (10.0, 100.0), 1, 0.15),
    "large8_256x1024": (8, 100.0, 256, {1024}, (120.0, 120.0), 1, 0.15),
    "paper_L39_64x64": (1, 39.0, 64, {64}, (40.0, 40.0), 1, 0.15),
    "paper_L39_xi_64x64": (1, 39.0, 64, {64}, (40.0, 40.0), 1, 0.15),
}


@pytest.mark.parametrize("name", inputs.WORKLOADS)
def test_workload_configuration(name):
    w = inputs.workload(name)
    B, L, nx, nsset, (lo, hi), scheme, dtau = EXPECTED[name]
    assert w.batch == B and w.L == L and w.nx == nx and w.scheme == scheme and w.dtau == dtau
    assert set(w.ns) <= nsset and all(lo <= T <= hi for T in w.T0)
    if name == "ragged256_64xNs":
        assert set(w.ns) == nsset                     # every length occurs
    assert w.packed().size == sum(w.ns) * nx


@pytest.mark.parametrize("name", ["single_64x128_imex", "batch16_64x64", "paper_L39_xi_64x64"])
def test_loops_follow_the_recipe(name):
    w = inputs.workload(name)
    again = inputs.workload(name)
    for b, u in enumerate(w.u):
        ns, nx = u.shape
        assert np.array_equal(u, again.u[b])                     # seeded
        assert abs(u.mean()) < 1e-12 and abs(np.sqrt((u * u).mean()) - 1.0) < 1e-12
        c = np.fft.fft2(u) / u.size                                # test-side spectrum check
        k = np.fft.fftfreq(ns, 1.0 / ns)[:, None]
        j = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
        outside = (np.abs(j) > nx // 3) | (np.abs(k) > ns // 3)
        assert np.abs(c[outside]).max() < 1e-13
        assert np.abs(c[:, 0]).max() < 1e-13                        # j = 0 column zeroed
        if name.startswith("paper_L39_xi"):
            assert np.abs(u + np.roll(u[:, ::-1], 1, axis=1)).max() < 1e-12   # odd in x


def test_stored_orbit_guess_is_a_centre_symmetric_recurrence_loop():
    """The stored loop at the paper's setting: 64 x 64 at L = 39, band limited, odd in x, a
    period in the recurrence range, and far closer to a solution than a random loop of the same
    size (its J, evaluated by the oracle, is a small fraction of its energy)."""
    import math
    from oracle import ks_oracle as ko
    from paper_2007_06427_gb300.inputs import orbit_guess
    w = orbit_guess()
    assert (w.L, w.nx, w.ns, w.batch) == (39.0, 64, [64], 1)
    assert 20.0 <= w.T0[0] <= 32.0
    u = w.u[0]
    g = ko.grid(64, 64, 39.0)
    spec = g.to_spectral(u)
    assert np.abs(np.where(g.mask, 0, spec)).max() < 1e-13 * np.abs(spec).max()
    assert np.abs(u + np.roll(u[:, ::-1], 1, axis=1)).max() < 1e-13 * np.abs(u).max()
    J = ko.residual(u, w.T0[0], w.L, xi=True)["J"]
    e = w.L * np.mean(u * u)
    rnd, _, _ = spectral_loop(0, 64, 39.0, ns=64, T0=w.T0[0], symmetric=True)
    J_rnd = ko.residual(rnd * math.sqrt(np.mean(u * u)), w.T0[0], w.L, xi=True)["J"]
    assert J / e < 0.03 and J < 0.05 * J_rnd, (J / e, J / J_rnd)   # measured 0.0099, 0.017
