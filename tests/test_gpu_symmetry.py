"""GPU: the descent restricted to the centre-symmetric subspace (the "symmetry" knob).

A loop is Xi-invariant when u(-x, s) = -u(x, s) (Eq. KS_loop_sym); the paper's initial loops and
orbits all are (Sec. 4.4).  With the knob set, every analysis of a grid field and every descent
direction is projected onto that subspace.  Checked here against the oracle's xi=True
evaluation (FP64 1e-12, FP32 1e-5 relative), bit-exact invariance of the band state
(u_hat[j][-k] = -conj(u_hat[j][k]), zero j = 0 column) on all three launch paths and in mixed
precision, bit-identical results across the paths, and that without the knob the flow keeps an
invariant loop invariant up to rounding (Sec. 4.1).
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


def make(nx, nss, L=22.0, symmetric=True, T_range=(20.0, 80.0)):
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i, nx, L, ns=n, T_range=T_range, symmetric=symmetric)
        us.append(u)
        Ts.append(T)
    return us, Ts


def dev(us, Ts, mode):
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).to("cuda", dt)
    return u, torch.tensor(Ts, dtype=torch.float64, device="cuda")


def split(flat, nx, nss):
    out, o = [], 0
    for n in nss:
        out.append(flat[o:o + n * nx].reshape(n, nx))
        o += n * nx
    return out


def band_violations(h, nx, nss):
    """Count band entries breaking u_hat[j][-k] == -conj(u_hat[j][k]) or a zero j = 0 column,
    compared bit for bit."""
    nb = K.ks_band_size(h.handle)
    band = torch.zeros(2 * nb, dtype=torch.float64, device="cuda")
    K.ks_get_band(h.handle, band)
    a = band.cpu().numpy().reshape(-1, 2)
    kx = nx // 3
    bad, o = 0, 0
    for n in nss:
        ks = n // 3
        nk = 2 * ks + 1
        blk = a[o:o + (kx + 1) * nk].reshape(kx + 1, nk, 2)
        o += (kx + 1) * nk
        bad += int(np.count_nonzero(blk[0]))
        mir = blk[1:, ::-1, :]
        bad += int(np.count_nonzero(blk[1:, :, 0] != -mir[:, :, 0]))
        bad += int(np.count_nonzero(blk[1:, :, 1] != mir[:, :, 1]))
    assert o == nb
    return bad


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
@pytest.mark.parametrize("symmetric", [True, False])
def test_residual_and_gradient_in_subspace(mode, symmetric):
    """r, G (projected), J, dJ/dT of P_Xi P u against the oracle; a non-invariant input is
    projected first."""
    L, nx, nss = 22.0, 64, [32, 64, 128]
    us, Ts = make(nx, nss, L, symmetric)
    if mode == K.KS_FP32:
        us = [a.astype(np.float32).astype(np.float64) for a in us]
    u, T = dev(us, Ts, mode)
    with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15) as h:
        K.ks_set_option(h.handle, "symmetry", 1)
        assert K.ks_get_option(h.handle, "symmetry") == 1
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
        ref = ko.adjoint_grad(us[b], Ts[b], L, xi=True)
        assert rel(rs[b], ko.residual(us[b], Ts[b], L, xi=True)["r"]) < tol
        assert rel(Gs[b], ref["G"]) < tol, (b, rel(Gs[b], ref["G"]))
        assert abs(J[b].item() - ref["J"]) <= tol * ref["J"]
        assert abs(dJdT[b].item() - ref["dJdT"]) <= tol * abs(ref["dJdT"]) + 1e-300


@pytest.mark.parametrize("symmetric", [True, False])
def test_descent_trajectory_in_subspace(symmetric):
    """20 IMEX steps in the subspace follow the oracle's projected descent (FP64, 1e-12)."""
    L, nx, nss, n = 22.0, 32, [32, 16, 64], 20
    us, Ts = make(nx, nss, L, symmetric)
    u, T = dev(us, Ts, K.KS_FP64)
    B = len(nss)
    sq = torch.zeros(B, dtype=torch.float64, device="cuda")
    with K.KSLoop(L, nx, nss, K.KS_FP64, K.KS_IMEX, 0.15, chunk=7) as h:
        K.ks_set_option(h.handle, "symmetry", 1)
        K.ks_descend(h.handle, u, T, n, 0.0, None, sq)
        assert band_violations(h, nx, nss) == 0
    out = split(u.cpu().numpy(), nx, nss)
    for b in range(B):
        d = ko.descend(us[b], Ts[b], L, 0.15, ko.IMEX, n, xi=True)
        assert rel(out[b], d["u"]) < 1e-12
        assert abs(T[b].item() - d["T"]) < 1e-12 * d["T"]
        assert abs(sq[b].item() - d["sqrtJ"]) < 1e-11 * d["sqrtJ"]


def test_fp32_descent_in_subspace():
    L, nx, nss, n = 22.0, 64, [64, 128], 30
    us, Ts = make(nx, nss, L)
    us = [a.astype(np.float32).astype(np.float64) for a in us]
    u, T = dev(us, Ts, K.KS_FP32)
    with K.KSLoop(L, nx, nss, K.KS_FP32, K.KS_IMEX, 0.15, chunk=11) as h:
        K.ks_set_option(h.handle, "symmetry", 1)
        K.ks_descend(h.handle, u, T, n, 0.0)
        assert band_violations(h, nx, nss) == 0
    out = split(u.double().cpu().numpy(), nx, nss)
    for b in range(len(nss)):
        d = ko.descend(us[b], Ts[b], L, 0.15, ko.IMEX, n, xi=True)
        assert rel(out[b], d["u"]) < 1e-5


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
def test_paths_bit_identical_in_subspace(mode):
    """Cluster-resident, persistent and per-phase launches agree bit for bit with the knob set,
    and each keeps the band exactly invariant."""
    L, nx, nss = 22.0, 64, [128, 32, 64, 256]
    us, Ts = make(nx, nss, L, symmetric=False)
    outs = []
    for path in (0, 1, 2):
        u, T = dev(us, Ts, mode)
        sq = torch.zeros(len(nss), dtype=torch.float64, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, chunk=6) as h:
            K.ks_set_option(h.handle, "path", path)
            K.ks_set_option(h.handle, "symmetry", 1)
            K.ks_descend(h.handle, u, T, 15, 0.0, None, sq)
            assert band_violations(h, nx, nss) == 0, path
        outs.append((u.cpu(), T.cpu(), sq.cpu()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


@pytest.mark.parametrize("C", [2, 16])
def test_cluster_sizes_in_subspace(C):
    L, nx, nss = 22.0, 64, [128]
    us, Ts = make(nx, nss, L)
    outs = []
    for path in (0, 2):
        u, T = dev(us, Ts, K.KS_FP64)
        with K.KSLoop(L, nx, nss, K.KS_FP64, K.KS_IMEX, 0.15, chunk=5) as h:
            K.ks_set_option(h.handle, "path", path)
            K.ks_set_option(h.handle, "symmetry", 1)
            if path == 0:
                K.ks_set_option(h.handle, "cluster", C)
                if K.ks_get_option(h.handle, "cluster_f64") != C:
                    pytest.skip(f"cluster size {C} does not fit")
            K.ks_descend(h.handle, u, T, 12, 0.0)
        outs.append((u.cpu(), T.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("f32_adjoint", [1, 0])
def test_mixed_descent_stays_invariant(f32_adjoint):
    """Float bulk, then double finish, in the subspace: the band is exactly invariant after the
    switch and the converged state matches the class of a plain FP64 descent's."""
    L, nx, nss = 22.0, 32, [32, 64]
    us, Ts = make(nx, nss, L, T_range=(30.0, 50.0))
    us = [1e-2 * a for a in us]
    u, T = dev(us, Ts, K.KS_FP64)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    sq = torch.zeros(2, dtype=torch.float64, device="cuda")
    with K.KSLoop(L, nx, nss, K.KS_MIXED, K.KS_IMEX, 0.15, tol=1e-10, switch_tol=1e-6,
                  chunk=2000) as h:
        K.ks_set_option(h.handle, "symmetry", 1)
        K.ks_set_option(h.handle, "finish_f32_adjoint", f32_adjoint)
        K.ks_descend(h.handle, u, T, 400000, 1e-10, None, sq, st)
        assert band_violations(h, nx, nss) == 0
        hs, hq, hp = K.ks_get_history(h.handle, 0)
        assert hp[0] == 1 and hp[-1] == 0
    assert st.tolist() == [K.KS_CONVERGED] * 2
    for a in split(u.cpu().numpy(), nx, nss):
        # u odd in x has zero mean: the invariant equilibrium reached is u = 0
        assert np.abs(a).max() < 1e-6


def test_flow_preserves_symmetry_without_projection():
    """Without the knob an invariant loop stays invariant up to rounding (Sec. 4.1): after 300
    IMEX steps the non-invariant part of the band is at the rounding level."""
    L, nx, nss = 22.0, 64, [64]
    us, Ts = make(nx, nss, L)
    u, T = dev(us, Ts, K.KS_FP64)
    with K.KSLoop(L, nx, nss, K.KS_FP64, K.KS_IMEX, 0.15, chunk=100) as h:
        K.ks_descend(h.handle, u, T, 300, 0.0)
    a = u.cpu().numpy().reshape(nss[0], nx)
    odd_part = 0.5 * (a - np.roll(a[:, ::-1], 1, axis=1))
    assert np.abs(a - odd_part).max() < 1e-10 * np.abs(a).max()


def test_extrapolated_descent_stays_invariant():
    """The extrapolation of App. C inside ks_descend moves a loop along a combination of two
    invariant states, so with the knob set the band stays exactly invariant through it."""
    L, nx, nss = 22.0, 32, [32, 64]
    us, Ts = make(nx, nss, L, T_range=(30.0, 50.0))
    us = [1e-2 * a for a in us]
    u, T = dev(us, Ts, K.KS_FP64)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    with K.KSLoop(L, nx, nss, K.KS_MIXED, K.KS_IMEX, 0.15, tol=1e-10, switch_tol=1e-6,
                  chunk=500) as h:
        K.ks_set_option(h.handle, "symmetry", 1)
        K.ks_set_option(h.handle, "extrapolate", 1)
        K.ks_descend(h.handle, u, T, 400000, 1e-10, None, None, st)
        assert K.ks_get_option(h.handle, "extrapolations") >= 1
        assert band_violations(h, nx, nss) == 0
    assert st.tolist() == [K.KS_CONVERGED] * 2
