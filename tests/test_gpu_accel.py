"""Extrapolation along the leading eigendirection (App. C): same fixed point, fewer steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.accel import descend_extrapolated
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu


def test_extrapolation_converges_with_fewer_steps():
    L, nx, ns = 22.0, 32, 32
    u0, T0, _ = spectral_loop(2, nx, L, ns=ns, T_range=(30.0, 50.0))
    u0 = 1e-2 * u0                      # small loop: the constant equilibria attract it
    u = torch.tensor(u0.ravel(), device="cuda")
    with K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15) as h:
        plain = descend_extrapolated(h, u, T0, tol=1e-10, start=0.0, chunk=200)
        acc = descend_extrapolated(h, u, T0, tol=1e-10, start=1e-3, chunk=200)
    assert plain.status == K.KS_CONVERGED and acc.status == K.KS_CONVERGED
    assert plain.extrapolations == 0
    assert acc.extrapolations >= 1
    assert acc.sqrtJ < 1e-10
    assert acc.steps < 0.7 * plain.steps, (acc.steps, plain.steps)
    # same class of fixed point: the fluctuation has decayed in both
    for r in (plain, acc):
        a = r.u.cpu().numpy().reshape(ns, nx)
        assert np.abs(a - a.mean()).max() < 1e-6


def test_mixed_extrapolation_converges():
    """Float bulk and double finish, both extrapolated: converges below 1e-10 to the same class
    of fixed point, with at least one kept extrapolation and a switch to double."""
    from paper_2007_06427_gb300.accel import descend_extrapolated_mixed
    L, nx, ns = 22.0, 32, 32
    u0, T0, _ = spectral_loop(2, nx, L, ns=ns, T_range=(30.0, 50.0))
    u0 = 1e-2 * u0
    u = torch.tensor(u0.ravel(), device="cuda")
    with K.KSLoop(L, nx, [ns], K.KS_FP32, K.KS_IMEX, 0.15) as h32, \
            K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15) as h64:
        r = descend_extrapolated_mixed(h32, h64, u, T0, tol=1e-10, chunk=200)
        plain = descend_extrapolated(h64, u, T0, tol=1e-10, start=0.0, chunk=200)
    assert r.status == K.KS_CONVERGED and r.sqrtJ < 1e-10
    assert r.switch_step is not None and r.extrapolations >= 1
    assert r.steps < plain.steps
    a = r.u.cpu().numpy().reshape(ns, nx)
    assert np.abs(a - a.mean()).max() < 1e-6
    # in the double phase the recorded sqrt(J) never increases from one kept state to the next
    after = [s for st, s, ev in r.history if st >= r.switch_step and ev != "rejected"]
    assert len(after) >= 2
    assert all(b <= a * (1 + 1e-9) for a, b in zip(after, after[1:]))


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
