"""The GPU integrator of the KSE and the initial-loop pipeline (Sec. 4.3) through the C ABI
(``ks_dns``, ``ks_dns_segments``) against the oracle (``ko.dns``, ``ko.segment_loop``,
``ko.norm_series``), and the properties that hold at any size: the linear symbol, the conserved
mean, fourth-order convergence, the right-hand side of the KSE, the centre-symmetric subspace.

Tolerance of the run against the oracle: both integrate the same semi-discrete system in FP64 and
differ by transform rounding (~1e-15 per step); a chaotic run amplifies that difference
exponentially, so the comparison is over a short horizon (t <= 50, growth below 1e3) at 1e-11 of
the field's largest value."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ks_oracle as ko
from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.guesses import chaotic_run, ks_dns, recurrence_loops

pytestmark = pytest.mark.gpu


def seeded_fields(L, nx, batch, seed, symmetric=False):
    """Seeded smooth fields of rms ~0.5: random coefficients on |j| <= 6 with e^{-j/2} decay."""
    rng = np.random.default_rng(seed)
    x = L * np.arange(nx) / nx
    out = np.zeros((batch, nx))
    for b in range(batch):
        for j in range(1, 7):
            q = 2 * math.pi * j / L
            a, c = rng.standard_normal(2) * math.exp(-j / 2)
            out[b] += a * np.sin(q * x) + (0.0 if symmetric else c * np.cos(q * x))
    return out


@pytest.mark.parametrize("L,nx,batch,dt,nsteps,every,sym", [
    (22.0, 64, 1, 0.25, 200, 50, False),     # the chaotic regime of the descent's domain
    (39.0, 64, 3, 0.25, 200, 40, True),      # the paper's domain, centre-symmetric, a pair + a ghost
    (22.0, 32, 9, 0.25, 120, 30, False),     # several blocks of four pairs
    (100.0, 256, 2, 0.1, 150, 50, False),    # a larger domain: one pair per block
])
def test_run_matches_oracle(L, nx, batch, dt, nsteps, every, sym):
    u0 = seeded_fields(L, nx, batch, seed=nx + batch, symmetric=sym)
    run = ks_dns(L, nx, dt, nsteps, u0, save_every=every, symmetric=sym)
    us = run.us.cpu().numpy()
    assert us.shape == (batch, nsteps // every + 1, nx)
    np.testing.assert_array_equal(run.ts, dt * every * np.arange(nsteps // every + 1))
    for b in range(batch):
        ts, ref = ko.dns(L, nx, dt, nsteps, u0[b], save_every=every, symmetric=sym)
        scale = np.abs(ref).max()
        assert np.abs(us[b] - ref).max() < 1e-11 * scale, (b, np.abs(us[b] - ref).max() / scale)
        np.testing.assert_allclose(run.norms[b], ko.norm_series(ref, L), rtol=1e-11, atol=0)


def test_end_state_zero_steps_and_host_buffers():
    """u_end is the state after the last step (saved or not); nsteps = 0 saves the projected
    initial field; host buffers give the same bits as device buffers."""
    L, nx, batch = 22.0, 32, 3
    u0 = seeded_fields(L, nx, batch, seed=7)
    dev = torch.tensor(u0, device="cuda")
    nsave = 45 // 10 + 1
    us = torch.empty(batch, nsave, nx, dtype=torch.float64, device="cuda")
    nrm = torch.empty(batch, nsave, dtype=torch.float64, device="cuda")
    end = torch.empty(batch, nx, dtype=torch.float64, device="cuda")
    K.ks_dns(L, nx, batch, 0.25, 45, 10, False, dev, us, nrm, end)
    torch.cuda.synchronize()
    h_us = np.empty((batch, nsave, nx))
    h_nrm = np.empty((batch, nsave))
    h_end = np.empty((batch, nx))
    K.ks_dns(L, nx, batch, 0.25, 45, 10, False, np.ascontiguousarray(u0), h_us, h_nrm, h_end)
    assert np.array_equal(h_us, us.cpu().numpy()) and np.array_equal(h_end, end.cpu().numpy())
    assert np.array_equal(h_nrm, nrm.cpu().numpy())
    for b in range(batch):
        _, ref = ko.dns(L, nx, 0.25, 45, u0[b], save_every=45)
        assert np.abs(h_end[b] - ref[-1]).max() < 1e-12 * np.abs(ref).max()
    zero = ks_dns(L, nx, 0.25, 0, u0[0], save_every=3)
    proj = ko.dns(L, nx, 0.25, 0, u0[0])[1]
    assert zero.us.shape == (1, nx)
    np.testing.assert_allclose(zero.us.cpu().numpy(), proj, rtol=0, atol=1e-14 * np.abs(proj).max())


@pytest.mark.parametrize("j", [1, 2, 3])
def test_linear_mode_follows_the_symbol(j):
    """ETDRK4 integrates the linear part exactly: a mode of amplitude 1e-12 (product ~1e-24)
    grows or decays by exp((q^2 - q^4) t)."""
    L, nx = 22.0, 32
    x = L * np.arange(nx) / nx
    q = 2 * math.pi * j / L
    run = ks_dns(L, nx, 0.25, 40, 1e-12 * np.cos(q * x), save_every=40)
    exact = 1e-12 * math.exp((q * q - q ** 4) * 10.0) * np.cos(q * x)
    np.testing.assert_allclose(run.us[-1].cpu().numpy(), exact, rtol=0, atol=1e-9 * np.abs(exact).max())


def test_mean_conserved_and_run_bounded():
    run = chaotic_run(22.0, 32, 400.0, seed=1)
    us = run.us.cpu().numpy()
    means = us.mean(axis=1)
    assert np.abs(means - means[0]).max() < 1e-13
    assert np.isfinite(run.norms).all() and 1.0 < run.norms[-200:].mean() < 30.0


def test_fourth_order_on_a_chaotic_state():
    """Halving dt divides the error at t = 1 by a factor approaching 2^4 = 16 (a scheme of order
    three or two would approach 8 or 4); reference: dt = 1/2048."""
    L, nx = 22.0, 64
    u0 = chaotic_run(L, nx, 300.0, seed=1).us[-1].cpu().numpy()

    def run(dt):
        n = int(round(1.0 / dt))
        return ks_dns(L, nx, dt, n, u0, save_every=n).us[-1].cpu().numpy()

    ref = run(1.0 / 2048)
    errs = [np.abs(run(dt) - ref).max() for dt in (1 / 64, 1 / 128, 1 / 256)]
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert ratios[1] > ratios[0] > 11.0, ratios
    assert math.log2(ratios[1]) > 3.7, ratios


def test_time_derivative_is_the_ks_right_hand_side():
    """The centred difference in time of the run on a chaotic state equals the oracle's
    right-hand side -u u_x - u_xx - u_xxxx of the same snapshot (the residual of a loop constant
    in s).  Second order in h: ~1.5e-7 at h = 1e-4."""
    L, nx, h = 22.0, 64, 1e-4
    u0 = chaotic_run(L, nx, 300.0, seed=1).us[-1].cpu().numpy()
    fine = ks_dns(L, nx, h / 8, 16, u0, save_every=8).us.cpu().numpy()   # u(0), u(h), u(2h)
    dudt = (fine[2] - fine[0]) / (2 * h)
    N = ko.residual(np.repeat(fine[1][None, :], 8, axis=0), 40.0, L)["r"][0]
    assert np.abs(dudt - N).max() < 1e-6 * np.abs(N).max()


def _reflect(u):
    """u(-x) on the grid x_m = m L / Nx (last axis)."""
    return np.roll(u[..., ::-1], 1, axis=-1)


def test_symmetric_run_and_loops_stay_centre_symmetric():
    """In the centre-symmetric subspace (Sec. 4.4) the run stays odd in x and chaotic, and the
    extracted loops are odd in x as well (L = 39, the paper's domain)."""
    L, nx, ns = 39.0, 64, 64
    run = chaotic_run(L, nx, 1500.0, seed=2, symmetric=True)
    us = run.us.cpu().numpy()
    assert np.abs(us + _reflect(us)).max() < 1e-13 * np.abs(us).max()
    tail = run.norms[-400:]
    assert np.isfinite(run.norms).all() and tail.mean() > 1.0 and np.ptp(tail) > 0.05 * tail.mean()
    loops = recurrence_loops(run, L, ns, T_range=(10.0, 120.0), tol=0.01, t_min=200.0, max_loops=2)
    assert len(loops) >= 1
    for lp in loops:
        assert np.abs(lp.u + _reflect(lp.u)).max() < 1e-12 * np.abs(lp.u).max()
        np.testing.assert_allclose(ko.band_state(lp.u, L, xi=True), ko.band_state(lp.u, L),
                                   rtol=0, atol=1e-13 * np.abs(lp.u).max())


def test_segments_match_oracle():
    """The segment cut through the C ABI against the oracle's linear interpolation, on the
    samples of a GPU run (the same input for both), for loops of several Ns, starts and periods;
    a segment past the saved samples is rejected."""
    L, nx = 22.0, 32
    run = chaotic_run(L, nx, 300.0, seed=3)
    us = run.us
    host = us.cpu().numpy()
    dts = float(run.ts[1] - run.ts[0])
    a_idx = [10, 250, 400, 3]
    Ts = [23.7, 41.25, 12.0, 80.3]
    nss = [32, 64, 16, 128]
    out = torch.empty(sum(n * nx for n in nss), dtype=torch.float64, device="cuda")
    K.ks_dns_segments(nx, host.shape[0], dts, us, a_idx, Ts, nss, out)
    got = out.cpu().numpy()
    o = 0
    for a, T, n in zip(a_idx, Ts, nss):
        ref = ko.segment_loop(run.ts, host, a, T, n)
        blk = got[o:o + n * nx].reshape(n, nx)
        assert np.abs(blk - ref).max() <= 1e-13 * np.abs(ref).max()
        o += n * nx
    with pytest.raises(K.KsError) as e:
        K.ks_dns_segments(nx, host.shape[0], dts, us, [host.shape[0] - 20], [50.0], [32], out)
    assert e.value.code == K.KS_ERR_ARG


def test_recurrence_loops_match_oracle():
    """The loops of the pipeline (pairs from the kernel's norm series, segment cut and band
    projection on the GPU) against the oracle's cut of the same samples, projected onto the band
    by the oracle: band limited and within 1e-12."""
    L, nx, ns = 22.0, 32, 32
    run = chaotic_run(L, nx, 2000.0, seed=0)
    loops = recurrence_loops(run, L, ns, T_range=(10.0, 80.0), tol=0.005, t_min=200.0, max_loops=3)
    assert len(loops) >= 1
    host = run.us.cpu().numpy()
    g = ko.grid(nx, ns, L)
    for lp in loops:
        a = int(np.argmin(np.abs(run.ts - lp.t0)))
        assert 10.0 <= lp.T <= 80.0 and lp.mismatch < 0.005
        ref = g.real_grid(ko.band_state(ko.segment_loop(run.ts, host, a, lp.T, ns), L))
        assert np.abs(lp.u - ref).max() < 1e-12 * np.abs(ref).max()
        spec = g.to_spectral(lp.u)
        assert np.abs(np.where(g.mask, 0, spec)).max() < 1e-12 * np.abs(spec).max()


def test_recurrence_loops_lie_near_solutions():
    """Loops from recurrences are far closer to solutions than random loops of the same size."""
    from paper_2007_06427_gb300.inputs import spectral_loop
    L, nx, ns = 22.0, 32, 32
    run = chaotic_run(L, nx, 2000.0, seed=0)
    loops = recurrence_loops(run, L, ns, T_range=(10.0, 80.0), tol=0.005, t_min=200.0, max_loops=3)
    rnd, _, _ = spectral_loop(0, nx, L, ns=ns, T0=40.0)
    for lp in loops:
        e = L * np.mean(lp.u ** 2)
        J = ko.residual(lp.u, lp.T, L)["J"]
        J_rnd = ko.residual(rnd * math.sqrt(np.mean(lp.u ** 2)), lp.T, L)["J"]
        assert J / e < 0.2 and J < 0.1 * J_rnd


def test_segments_reject_device_tables():
    """The per-loop tables are read on the host: device pointers there are rejected with
    KS_ERR_ARG (called through ctypes, since the binding always passes host arrays)."""
    import ctypes
    lib = K.load_library()
    us = torch.zeros(10, 8, dtype=torch.float64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    a_dev = torch.zeros(1, dtype=torch.int32, device="cuda")
    T = np.array([3.0])
    ns = np.array([8], dtype=np.int32)
    rc = lib.ks_dns_segments(8, 10, 0.5, ctypes.c_void_p(us.data_ptr()), 1, ctypes.c_void_p(a_dev.data_ptr()),
                             T.ctypes.data_as(ctypes.c_void_p), ns.ctypes.data_as(ctypes.c_void_p),
                             ctypes.c_void_p(out.data_ptr()), None)
    assert rc == K.KS_ERR_ARG
