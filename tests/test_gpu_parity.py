"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle, element by element.

Tolerances: FP64 mode 1e-12 relative (||x_gpu - x_oracle|| / ||x_oracle|| over each loop) on
r and G and on J, dJ/dT; FP32 mode 1e-5 relative.  An FP32 handle receives the field rounded
to float, so the oracle is given exactly those rounded values (in double): the comparison
measures the kernel's arithmetic, not the rounding of the input.  Shapes cover every workload's (Nx, Ns)
plus tiny and ragged batches (several transform tiles, ragged row tiles, loops of unequal Ns).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ks_oracle as ko
from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu

TOL = {K.KS_FP64: 1e-12, K.KS_FP32: 1e-5}


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def make(nx, nss, L=22.0, seed0=0, T_range=(20.0, 80.0), decay=(2.0, 2.0)):
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(seed0 + i, nx, L, ns=n, T_range=T_range, decay=decay)
        us.append(u)
        Ts.append(T)
    return us, Ts


def dev_tensors(us, Ts, mode):
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).to("cuda", dt)
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda")
    return u, T


def split(flat, nx, nss):
    out, o = [], 0
    for n in nss:
        out.append(flat[o:o + n * nx].reshape(n, nx))
        o += n * nx
    return out


SHAPES = [
    (32, [32]),                 # single 32 x 32 explicit workload
    (64, [128]),                # single 64 x 128 workload
    (64, [64, 64, 64]),         # batch of 64 x 64 loops
    (64, [32, 64, 128, 256]),   # ragged Ns
    (8, [8]),                   # smallest transform
    (16, [8, 16, 32]),          # ragged, odd log2 lengths
    (128, [16]),                # with L = 44: same q_max as Nx = 64 at L = 22
]


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
@pytest.mark.parametrize("nx,nss", SHAPES)
def test_residual_and_gradient_match_oracle(nx, nss, mode):
    # keep the largest retained wavenumber near the workloads' (q_max ~ 6, L = 22 Nx / 64) and
    # let the init spectrum reach the band edge as the workloads' do (decay ~ Kx / 10): bands
    # that extend far beyond the spectrum amplify FP64 rounding noise by the q^8 symbol of G
    # in any FP64 evaluation, the oracle's included
    L = 22.0 * max(1.0, nx / 64)
    dx = max(2.0, (nx // 3) / 10.0)
    us, Ts = make(nx, nss, L, decay=(dx, 2.0))
    if mode == K.KS_FP32:
        us = [a.astype(np.float32).astype(np.float64) for a in us]
    u, T = dev_tensors(us, Ts, mode)
    with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15) as h:
        r = torch.empty_like(u)
        G = torch.empty_like(u)
        J = torch.empty(len(nss), dtype=torch.float64, device="cuda")
        dJdT = torch.empty_like(J)
        K.ks_residual(h.handle, u, T, r, J)
        K.ks_adjoint_grad(h.handle, u, T, G, dJdT)
        torch.cuda.synchronize()
    rs = split(r.double().cpu().numpy(), nx, nss)
    Gs = split(G.double().cpu().numpy(), nx, nss)
    tol = TOL[mode]
    for b in range(len(nss)):
        ref = ko.adjoint_grad(us[b], Ts[b], L)
        r_ref = ko.grid(nx, nss[b], L).real_grid(ref["rh"])
        assert rel(rs[b], r_ref) < tol, (b, rel(rs[b], r_ref))
        assert rel(Gs[b], ref["G"]) < tol, (b, rel(Gs[b], ref["G"]))
        assert abs(J[b].item() - ref["J"]) <= tol * ref["J"]
        assert abs(dJdT[b].item() - ref["dJdT"]) <= tol * abs(ref["dJdT"]) + 1e-300


def test_large_domain_sampled():
    """256 x 1024 at L = 100 (the large-domain workload's shape): full r and G of one loop."""
    L, nx, ns = 100.0, 256, 1024
    us, Ts = make(nx, [ns], L, T_range=(120.0, 120.0), decay=(8.0, 8.0))
    u, T = dev_tensors(us, Ts, K.KS_FP64)
    with K.KSLoop(L, nx, [ns], K.KS_FP64) as h:
        G = torch.empty_like(u)
        dJdT = torch.empty(1, dtype=torch.float64, device="cuda")
        K.ks_adjoint_grad(h.handle, u, T, G, dJdT)
        torch.cuda.synchronize()
    ref = ko.adjoint_grad(us[0], Ts[0], L)
    assert rel(G.cpu().numpy().reshape(ns, nx), ref["G"]) < 1e-12
    assert abs(dJdT.item() - ref["dJdT"]) <= 1e-12 * abs(ref["dJdT"])


@pytest.mark.parametrize("scheme,dtau,nsteps", [(K.KS_IMEX, 0.15, 20), (K.KS_EXPLICIT, 1e-4, 50)])
def test_descent_trajectory_matches_oracle(scheme, dtau, nsteps):
    L, nx, nss = 22.0, 32, [32, 16, 64]
    us, Ts = make(nx, nss, L)
    u, T = dev_tensors(us, Ts, K.KS_FP64)
    B = len(nss)
    steps = torch.zeros(B, dtype=torch.int64, device="cuda")
    sq = torch.zeros(B, dtype=torch.float64, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    with K.KSLoop(L, nx, nss, K.KS_FP64, scheme, dtau, chunk=7) as h:
        K.ks_descend(h.handle, u, T, nsteps, 0.0, steps, sq, st)
    us_out = split(u.cpu().numpy(), nx, nss)
    for b in range(B):
        d = ko.descend(us[b], Ts[b], L, dtau, scheme, nsteps)
        assert rel(us_out[b], d["u"]) < 1e-12
        assert abs(T[b].item() - d["T"]) < 1e-12 * d["T"]
        assert abs(sq[b].item() - d["sqrtJ"]) < 1e-11 * d["sqrtJ"]
        assert int(steps[b]) == nsteps
        assert int(st[b]) == K.KS_STEP_CAP


def test_explicit_2000_steps_single_32x32():
    """The 32 x 32 explicit workload: 2000 steps at dtau = 1e-4 against the oracle."""
    L, nx = 22.0, 32
    u0, T0, _ = spectral_loop(0, nx, L, ns=32, T0=40.0)
    u, T = dev_tensors([u0], [T0], K.KS_FP64)
    with K.KSLoop(L, nx, [32], K.KS_FP64, K.KS_EXPLICIT, 1e-4, chunk=500) as h:
        sq = torch.zeros(1, dtype=torch.float64, device="cuda")
        K.ks_descend(h.handle, u, T, 2000, 0.0, None, sq, None)
    d = ko.descend(u0, T0, L, 1e-4, ko.EXPLICIT, 2000)
    assert rel(u.cpu().numpy().reshape(32, 32), d["u"]) < 1e-11
    assert abs(T.item() - d["T"]) < 1e-12 * d["T"]
    assert sq.item() == pytest.approx(d["sqrtJ"], rel=1e-10)


def test_fp32_descent_tracks_oracle():
    L, nx, nss = 22.0, 64, [64, 128]
    us, Ts = make(nx, nss, L)
    us = [a.astype(np.float32).astype(np.float64) for a in us]
    u, T = dev_tensors(us, Ts, K.KS_FP32)
    with K.KSLoop(L, nx, nss, K.KS_FP32, K.KS_IMEX, 0.15) as h:
        K.ks_descend(h.handle, u, T, 10, 0.0)
    us_out = split(u.double().cpu().numpy(), nx, nss)
    for b in range(len(nss)):
        d = ko.descend(us[b], Ts[b], L, 0.15, ko.IMEX, 10)
        assert rel(us_out[b], d["u"]) < 1e-5
        assert abs(T[b].item() - d["T"]) < 1e-5 * d["T"]


def test_host_buffers_match_device_buffers():
    L, nx, nss = 22.0, 32, [32, 64]
    us, Ts = make(nx, nss, L)
    u, T = dev_tensors(us, Ts, K.KS_FP64)
    uh = np.concatenate([a.ravel() for a in us])
    Th = np.array(Ts)
    with K.KSLoop(L, nx, nss, K.KS_FP64) as h:
        G_d = torch.empty_like(u)
        K.ks_adjoint_grad(h.handle, u, T, G_d)
        G_h = np.empty_like(uh)
        dJ_h = np.empty(2)
        K.ks_adjoint_grad(h.handle, uh, Th, G_h, dJ_h)
        st_h = np.zeros(2, dtype=np.int32)
        K.ks_descend(h.handle, uh, Th, 5, 0.0, None, None, st_h)
        K.ks_descend(h.handle, u, T, 5, 0.0)
    np.testing.assert_array_equal(G_h, G_d.cpu().numpy())
    np.testing.assert_array_equal(uh, u.cpu().numpy())
    np.testing.assert_array_equal(Th, T.cpu().numpy())
    assert list(st_h) == [K.KS_STEP_CAP] * 2


def test_resident_state_steps_equal_descend():
    L, nx, nss = 22.0, 64, [64, 32]
    us, Ts = make(nx, nss, L)
    u, T = dev_tensors(us, Ts, K.KS_FP64)
    with K.KSLoop(L, nx, nss, K.KS_FP64) as h:
        K.ks_set_state(h.handle, u, T)
        for _ in range(3):
            K.ks_step(h.handle, 4, 0.0)
        u1 = torch.empty_like(u)
        T1 = torch.empty_like(T)
        steps = torch.zeros(2, dtype=torch.int64, device="cuda")
        K.ks_get_state(h.handle, u1, T1, steps)
        u2, T2 = u.clone(), T.clone()
        K.ks_descend(h.handle, u2, T2, 12, 0.0)
    assert steps.tolist() == [12, 12]
    assert torch.equal(u1, u2) and torch.equal(T1, T2)


def test_converged_and_trivial_loops():
    """u = 0 is an equilibrium (J = 0): converged with zero steps; a loop with T = NaN diverges;
    the others keep running."""
    L, nx, nss = 22.0, 32, [32, 32, 32]
    us, Ts = make(nx, nss, L)
    us[0] = np.zeros_like(us[0])
    Ts[2] = float("nan")
    u, T = dev_tensors(us, Ts, K.KS_FP64)
    steps = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.zeros(3, dtype=torch.int32, device="cuda")
    with K.KSLoop(L, nx, nss, K.KS_FP64) as h:
        K.ks_descend(h.handle, u, T, 10, 1e-10, steps, None, st)
    assert st.tolist() == [K.KS_CONVERGED, K.KS_STEP_CAP, K.KS_DIVERGED]
    assert steps.tolist()[:2] == [0, 10]


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
def test_persistent_kernel_equals_phase_launches(mode):
    """One cooperative launch per chunk (grid barriers between phases) gives bit-identical
    results to four launches per tau-step."""
    L, nx, nss = 22.0, 64, [128, 32, 64]
    us, Ts = make(nx, nss, L)
    outs = []
    for persistent in (1, 0):
        u, T = dev_tensors(us, Ts, mode)
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, chunk=5) as h:
            K.ks_set_option(h.handle, "persistent", persistent)
            K.ks_descend(h.handle, u, T, 17, 0.0)
        outs.append((u.cpu(), T.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("f32_adjoint", [1, 0])
def test_mixed_descent_converges_and_switches(f32_adjoint):
    """FP32 bulk, then FP64 finish (with the adjoint half of each finishing step in float, or
    all in double): a small-amplitude loop descends to sqrt(J) < 1e-10 (the constant
    equilibria attract it); the result is in the same class as a plain FP64 descent's."""
    L, nx, nss = 22.0, 32, [32, 64]
    us, Ts = make(nx, nss, L, T_range=(30.0, 50.0))
    us = [1e-2 * a for a in us]
    res = {}
    for mode in (K.KS_FP64, K.KS_MIXED):
        u, T = dev_tensors(us, Ts, K.KS_FP64)
        steps = torch.zeros(2, dtype=torch.int64, device="cuda")
        sq = torch.zeros(2, dtype=torch.float64, device="cuda")
        st = torch.zeros(2, dtype=torch.int32, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, tol=1e-10, switch_tol=1e-6,
                      chunk=2000) as h:
            if mode == K.KS_MIXED:
                K.ks_set_option(h.handle, "finish_f32_adjoint", f32_adjoint)
            K.ks_descend(h.handle, u, T, 400000, 1e-10, steps, sq, st)
            if mode == K.KS_MIXED:
                hs, hq, hp = K.ks_get_history(h.handle, 0)
                assert hp[0] == 1 and hp[-1] == 0      # float bulk, then double finish
                assert np.all(np.diff(hs) > 0)
        res[mode] = (u.cpu().numpy(), steps.tolist(), sq.tolist(), st.tolist(), T.cpu().numpy())
    for mode in (K.KS_FP64, K.KS_MIXED):
        u, steps, sq, st, _ = res[mode]
        assert st == [K.KS_CONVERGED] * 2, (mode, st, sq, steps)
        assert max(sq) < 1e-10
        # u = const is an equilibrium for every constant (Sec. 4.1): the mean may drift, the
        # fluctuation decays
        for a in split(u, nx, nss):
            assert np.abs(a - a.mean()).max() < 1e-6
    # the float bulk takes about as many steps as the double descent
    for b in range(2):
        assert abs(res[K.KS_MIXED][1][b] - res[K.KS_FP64][1][b]) < 0.2 * res[K.KS_FP64][1][b]


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
@pytest.mark.parametrize("nx,nss", [(64, [128]), (32, [32, 16, 64]), (64, [32, 64, 128, 256]),
                                    (16, [8])])
@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_cluster_kernel_equals_phase_launches(mode, nx, nss, C):
    """The cluster-resident kernel (one cluster of C CTAs per loop, distributed shared memory)
    reproduces the per-phase launches bit for bit, including across chunk boundaries."""
    L = 22.0
    us, Ts = make(nx, nss, L)
    outs = []
    for path in (0, 2):
        u, T = dev_tensors(us, Ts, mode)
        steps = torch.zeros(len(nss), dtype=torch.int64, device="cuda")
        sq = torch.zeros(len(nss), dtype=torch.float64, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, chunk=5) as h:
            K.ks_set_option(h.handle, "path", path)
            if path == 0:
                try:
                    K.ks_set_option(h.handle, "cluster", C)
                except K.KsError:
                    pytest.skip(f"cluster size {C} does not fit")
                key = "cluster_f32" if mode == K.KS_FP32 else "cluster_f64"
                if K.ks_get_option(h.handle, key) != C:
                    pytest.skip(f"cluster size {C} does not fit this precision")
            K.ks_descend(h.handle, u, T, 13, 0.0, steps, sq)
        outs.append((u.cpu(), T.cpu(), steps.cpu(), sq.cpu()))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_mixed_descent_starts_below_float_floor_in_double():
    """A loop already far below the float floor (a nontrivial KS equilibrium reached by a
    centre-symmetric run at L = 22, repeated over s): a mixed descent must not first raise its
    sqrt(J) to the float floor; it descends in double from the first chunk."""
    from paper_2007_06427_gb300.guesses import chaotic_run
    L, nx, ns = 22.0, 32, 32
    us = chaotic_run(L, nx, 1500.0, seed=0, symmetric=True).us
    loop = np.repeat(us[-1].cpu().numpy()[None, :], ns, axis=0)
    u = torch.tensor(loop.ravel(), device="cuda")
    T = torch.tensor([11.0], dtype=torch.float64, device="cuda")
    J0 = torch.empty(1, dtype=torch.float64, device="cuda")
    sq = torch.zeros(1, dtype=torch.float64, device="cuda")
    with K.KSLoop(L, nx, [ns], K.KS_MIXED, K.KS_IMEX, 0.15, chunk=2000) as h:
        K.ks_residual(h.handle, u, T, None, J0)
        K.ks_descend(h.handle, u, T, 20000, 1e-11, None, sq, None)
        hs, hq, hp = K.ks_get_history(h.handle, 0)
    assert np.sqrt(np.mean(loop ** 2)) > 0.5                 # nontrivial state
    assert np.sqrt(J0.item()) < 1e-6
    assert hp[0] == 0                                       # double from the first chunk
    assert sq.item() <= np.sqrt(J0.item())


def test_mixed_batch_concurrent_precisions_equal_sequential():
    """While a mixed batch has loops in both precisions, the float and double cluster launches
    run concurrently on two streams (each carrying T only for its own frozen loops).  With the
    library's profiling on they run one after the other; the results agree bit for bit."""
    L, nx, nss = 22.0, 32, [32, 32, 64, 32]
    us, Ts = make(nx, nss, L, T_range=(30.0, 50.0))
    us = [a * s for a, s in zip(us, (1e-2, 3e-3, 1e-2, 1.0))]   # loops that switch at different times
    outs = []
    for prof in (False, True):
        u, T = dev_tensors(us, Ts, K.KS_FP64)
        steps = torch.zeros(4, dtype=torch.int64, device="cuda")
        sq = torch.zeros(4, dtype=torch.float64, device="cuda")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        with K.KSLoop(L, nx, nss, K.KS_MIXED, K.KS_IMEX, 0.15, tol=1e-10, switch_tol=1e-5,
                      chunk=500) as h:
            K.ks_profile(h.handle, prof)
            K.ks_descend(h.handle, u, T, 60000, 1e-10, steps, sq, st)
            hp = [K.ks_get_history(h.handle, b)[2] for b in range(4)]
        outs.append((u.cpu(), T.cpu(), steps.cpu(), st.cpu()))
        # at some read-back one loop was in float while another was in double
        mixed_phase = any((hp[a][i] == 1) and (hp[b][i] == 0)
                          for a in range(4) for b in range(4)
                          for i in range(min(len(hp[a]), len(hp[b]))))
        assert mixed_phase
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_mixed_switch_probe_on_a_periodic_orbit():
    """The float-floor probe of a mixed descent (knob "switch_probe") on the stored recurrence
    loop at L = 39: the float phase of this loop stalls at sqrt(J) ~ 3e-5 with nothing converging
    beneath its noise, so the probe switches it to double soon after its rate bends and the loop
    converges below 1e-10 to the periodic orbit (T = 25.3708).  With the stall window alone the
    float phase runs on far longer (measured: switch at 524k steps, or 1.72M with the paired
    column transforms of the subspace), so within 600k steps it has switched much later or not
    at all, and has not converged."""
    from paper_2007_06427_gb300.inputs import orbit_guess
    w = orbit_guess()
    out = {}
    for probe, cap in ((1, 2_000_000), (0, 600_000)):
        u = torch.tensor(w.u[0].ravel(), device="cuda")
        T = torch.tensor(w.T0, dtype=torch.float64, device="cuda")
        steps = torch.zeros(1, dtype=torch.int64, device="cuda")
        sq = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        with K.KSLoop(w.L, w.nx, w.ns, K.KS_MIXED, K.KS_IMEX, 0.15, chunk=2000) as h:
            K.ks_set_option(h.handle, "symmetry", 1)
            assert K.ks_get_option(h.handle, "switch_probe") == 1
            assert K.ks_get_option(h.handle, "switch_probe_steps") == 1000
            K.ks_set_option(h.handle, "switch_probe", probe)
            K.ks_descend(h.handle, u, T, cap, 1e-10, steps, sq, st)
            hs, hq, hp = K.ks_get_history(h.handle, 0)
        sw = int(hs[np.nonzero(hp == 0)[0][0]]) if (hp == 0).any() else None
        out[probe] = (int(steps.item()), float(sq.item()), int(st.item()), float(T.item()), sw)
    n1, sq1, st1, T1, sw1 = out[1]
    assert st1 == K.KS_CONVERGED and sq1 < 1e-10 and abs(T1 - 25.3708) < 1e-3, out
    assert sw1 is not None and sw1 < 300_000, out
    n0, sq0, st0, T0, sw0 = out[0]
    assert st0 != K.KS_CONVERGED, out
    assert sw0 is None or sw0 > 2 * sw1, out
    with K.KSLoop(w.L, w.nx, w.ns, K.KS_MIXED) as h:
        for bad in (0, 1000001):
            with pytest.raises(K.KsError):
                K.ks_set_option(h.handle, "switch_probe_steps", bad)
