"""Extrapolation along the leading eigendirection (App. C): same fixed point, fewer steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu


def test_refine_uses_the_native_extrapolation():
    """orbits.refine (one loop, mixed precision, App. C inside ks_descend): converges below
    1e-10 to the same class of fixed point as the plain double descent, in fewer steps, with at
    least one kept extrapolation."""
    from paper_2007_06427_gb300.orbits import refine
    L, nx, ns = 22.0, 32, 32
    u0, T0, _ = spectral_loop(2, nx, L, ns=ns, T_range=(30.0, 50.0))
    u0 = 1e-2 * u0                      # small loop: the constant equilibria attract it
    r = refine(u0, T0, L, tol=1e-10, max_steps=400000, symmetric=False, chunk=200)
    u = torch.tensor(u0.ravel(), device="cuda")
    T = torch.tensor([T0], dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    with K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15, chunk=200) as h:
        K.ks_descend(h.handle, u, T, 400000, 1e-10, steps)
    assert r.status == K.KS_CONVERGED and r.sqrtJ < 1e-10
    assert r.extrapolations >= 1
    assert r.steps < int(steps.item()), (r.steps, int(steps.item()))
    for a in (r.u, u.cpu().numpy().reshape(ns, nx)):
        assert np.abs(a - a.mean()).max() < 1e-6


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_MIXED])
def test_native_extrapolation_in_batched_descent(mode):
    """The "extrapolate" knob of ks_descend (App. C inside the C driver): a batch of three loops
    converges below 1e-10 in fewer steps than the plain descent, to the same class of fixed
    point, and every loop of the batch follows the same path as when it descends alone."""
    L, nx, nss = 22.0, 32, [32, 32, 64]
    us, Ts = [], []
    for i, n in enumerate(nss):
        u0, T0, _ = spectral_loop(2 + i, nx, L, ns=n, T_range=(30.0, 50.0))
        us.append(1e-2 * u0)
        Ts.append(T0)

    def run(loops, extrap):
        idx = list(loops)
        u = torch.tensor(np.concatenate([us[b].ravel() for b in idx]), device="cuda")
        T = torch.tensor([Ts[b] for b in idx], dtype=torch.float64, device="cuda")
        steps = torch.zeros(len(idx), dtype=torch.int64, device="cuda")
        sq = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
        st = torch.zeros(len(idx), dtype=torch.int32, device="cuda")
        with K.KSLoop(L, nx, [nss[b] for b in idx], mode, K.KS_IMEX, 0.15, chunk=500,
                      switch_tol=1e-6) as h:
            K.ks_set_option(h.handle, "extrapolate", extrap)
            K.ks_descend(h.handle, u, T, 400000, 1e-10, steps, sq, st)
            nex = K.ks_get_option(h.handle, "extrapolations")
        return u.cpu().numpy(), T.cpu().numpy(), steps.tolist(), sq.tolist(), st.tolist(), nex

    plain = run(range(3), 0)
    acc = run(range(3), 1)
    assert acc[4] == [K.KS_CONVERGED] * 3 and max(acc[3]) < 1e-10
    assert acc[5] >= 3
    for b in range(3):
        assert acc[2][b] < 0.8 * plain[2][b], (acc[2], plain[2])
    o = 0
    for b in range(3):
        a = acc[0][o:o + nss[b] * nx]
        o += nss[b] * nx
        assert np.abs(a - a.mean()).max() < 1e-6
    # the loops of a batch do not influence each other
    alone = run([2], 1)
    assert alone[2][0] == acc[2][2] and alone[1][0] == acc[1][2]
    np.testing.assert_array_equal(alone[0], acc[0][2 * 32 * nx:])



def test_native_extrapolation_start_and_drop_knobs():
    """The start threshold and drop ratio of the native extrapolation: the defaults are the
    values of App. C's example (1e-3, halving); out-of-range values are refused; a drop ratio
    that is never reached leaves the descent plain (same steps and bits); an earlier start
    still converges, in fewer steps than the plain descent."""
    L, nx, ns = 22.0, 32, 32
    u0, T0, _ = spectral_loop(3, nx, L, ns=ns, T_range=(30.0, 50.0))
    u0 = 1e-2 * u0

    def run(**opts):
        u = torch.tensor(u0.ravel(), device="cuda")
        T = torch.tensor([T0], dtype=torch.float64, device="cuda")
        steps = torch.zeros(1, dtype=torch.int64, device="cuda")
        sq = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        with K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15, chunk=500) as h:
            assert K.ks_get_option(h.handle, "extrapolate_start_ppm") == 1000
            assert K.ks_get_option(h.handle, "extrapolate_drop_ppm") == 500000
            for k, v in opts.items():
                K.ks_set_option(h.handle, k, v)
                assert K.ks_get_option(h.handle, k) == v
            K.ks_descend(h.handle, u, T, 400000, 1e-10, steps, sq, st)
            nex = K.ks_get_option(h.handle, "extrapolations")
        return u.cpu().numpy(), float(T.item()), int(steps.item()), float(sq.item()), int(st.item()), nex

    with K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15) as h:
        for k, bad in (("extrapolate_start_ppm", 0), ("extrapolate_start_ppm", -5),
                       ("extrapolate_drop_ppm", 0), ("extrapolate_drop_ppm", 1000000)):
            with pytest.raises(K.KsError):
                K.ks_set_option(h.handle, k, bad)

    plain = run()
    # first anchor at sqrt(J) <= 1e-6, next move at <= 1e-12 of it: below the tolerance
    never = run(extrapolate=1, extrapolate_start_ppm=1, extrapolate_drop_ppm=1)
    assert never[5] == 0 and never[2] == plain[2] and never[1] == plain[1]
    np.testing.assert_array_equal(never[0], plain[0])
    base = run(extrapolate=1)
    early = run(extrapolate=1, extrapolate_start_ppm=100000)  # first anchor at sqrt(J) <= 0.1
    for r in (base, early):
        assert r[4] == K.KS_CONVERGED and r[3] < 1e-10 and r[5] >= 1
        assert r[2] < plain[2], (r[2], plain[2])


@pytest.mark.parametrize("seed,xi", [(3, False), (4, True)])
def test_native_extrapolation_matches_oracle(seed, xi):
    """ks_descend with the "extrapolate" knob against the oracle's App. C descent on the same
    loop and read-back schedule (every 100 steps): the same steps, the same extrapolations kept
    and rejected, and the final loop within the FP64 tolerance."""
    from oracle import ks_oracle as ko
    L, nx, ns = 22.0, 16, 16
    u0, T0, _ = spectral_loop(seed, nx, L, ns=ns, T_range=(30.0, 50.0), symmetric=xi)
    u0 = 1e-2 * u0
    ref = ko.descend_extrapolated(u0, T0, L, 0.15, ko.IMEX, 8000, 1e-10, 100, xi=xi)
    u = torch.tensor(u0.ravel(), device="cuda")
    T = torch.tensor([T0], dtype=torch.float64, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    sq = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15, chunk=100) as h:
        K.ks_set_option(h.handle, "extrapolate", 1)
        if xi:
            K.ks_set_option(h.handle, "symmetry", 1)
        K.ks_descend(h.handle, u, T, 8000, 1e-10, steps, sq, st)
        kept = K.ks_get_option(h.handle, "extrapolations")
        rejected = K.ks_get_option(h.handle, "extrapolations_rejected")
    assert int(st.item()) == K.KS_CONVERGED and ref["sqrtJ"] < 1e-10 and float(sq.item()) < 1e-10
    assert ref["extrapolations"] >= 3
    assert (int(steps.item()), kept, rejected) == (ref["steps"], ref["extrapolations"], ref["rejected"])
    ug = u.cpu().numpy().reshape(ns, nx)
    # measured against the larger of the final and the initial loop: the symmetric loop decays
    # to u = 0, where a relative error of the final field alone measures rounding noise
    scale = max(np.linalg.norm(ref["u"]), np.linalg.norm(u0))
    assert np.linalg.norm(ug - ref["u"]) <= 1e-12 * scale
    assert abs(float(T.item()) - ref["T"]) <= 1e-12 * abs(ref["T"])
