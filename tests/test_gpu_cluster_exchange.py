"""The cluster kernel's two exchange forms move the same values into the same buffers: stores
counted on the receiver's mbarrier (the default where the plan has room for the second column
buffer) or plain DSMEM stores separated by cluster barriers ("cluster_exchange" = 0).  A descent
therefore gives the same bits either way, on every column scheme and precision, including
clusters where some ranks own no columns or no rows.  The same holds for the kernel's two
launch-bound variants ("cluster_min_blocks"), which the plan picks by occupancy."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu

# (L, nx, loops' Ns, mode, centre-symmetric, switch_tol)
CASES = [
    (22.0, 64, [128], K.KS_FP64, False, 0.0),       # one loop, 16 ranks
    (22.0, 64, [128], K.KS_FP32, False, 0.0),
    (39.0, 64, [64] * 4, K.KS_FP64, True, 0.0),     # column pairs of the symmetric subspace
    (39.0, 64, [64] * 4, K.KS_FP32, True, 0.0),
    (22.0, 32, [32], K.KS_FP64, False, 0.0),        # 11 columns on 16 ranks
    (22.0, 32, [8], K.KS_FP32, False, 0.0),         # 8 rows on 16 ranks: most ranks own no row
    (22.0, 64, [64, 128, 32], K.KS_FP64, False, 0.0),  # ragged batch, one cluster per loop
    (22.0, 64, [64, 128], K.KS_MIXED, False, 1e6),  # switched at once: double state, float adjoint
]


def _loops(L, nx, nss, symmetric):
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(10 + i, nx, L, ns=n, T_range=(20.0, 80.0), symmetric=symmetric)
        us.append(u)
        Ts.append(T)
    return np.concatenate([a.ravel() for a in us]), Ts


@pytest.mark.parametrize("case", CASES, ids=[f"c{i}" for i in range(len(CASES))])
def test_exchange_forms_agree(case):
    L, nx, nss, mode, sym, swt = case
    u0, T0 = _loops(L, nx, nss, sym)
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    outs = []
    for xch in (1, 0):
        u = torch.tensor(u0, device="cuda").to(dt)
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, switch_tol=swt, chunk=7) as h:
            K.ks_set_option(h.handle, "path", 0)
            if sym:
                K.ks_set_option(h.handle, "symmetry", 1)
            if mode == K.KS_MIXED:
                K.ks_set_option(h.handle, "finish_f32_adjoint", 1)
            K.ks_set_option(h.handle, "cluster_exchange", xch)
            assert K.ks_get_option(h.handle, "cluster_exchange") == xch
            key = "cluster_exchange_f32" if mode == K.KS_FP32 else "cluster_exchange_f64"
            assert K.ks_get_option(h.handle, key) == xch  # these plans have room for it
            steps = torch.zeros(len(nss), dtype=torch.int64, device="cuda")
            K.ks_descend(h.handle, u, T, 20, 0.0, steps=steps)
            torch.cuda.synchronize()
            assert int(steps.min()) == 20
        outs.append((u.cpu(), T.cpu()))
    assert torch.isfinite(outs[0][0]).all()
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])


def _descend(L, nx, nss, mode, knobs, steps=20):
    u0, T0 = _loops(L, nx, nss, False)
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.tensor(u0, device="cuda").to(dt)
    T = torch.tensor(T0, dtype=torch.float64, device="cuda")
    with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, chunk=7) as h:
        K.ks_set_option(h.handle, "path", 0)
        for k, v in knobs.items():
            K.ks_set_option(h.handle, k, v)
        K.ks_descend(h.handle, u, T, steps, 0.0)
        torch.cuda.synchronize()
    return u.cpu(), T.cpu()


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
def test_launch_bound_variants_agree(mode):
    a = _descend(22.0, 64, [64] * 4, mode, {"cluster_min_blocks": 1})
    b = _descend(22.0, 64, [64] * 4, mode, {"cluster_min_blocks": 2})
    c = _descend(22.0, 64, [64] * 4, mode, {"cluster_min_blocks": 2, "cluster_exchange": 0})
    assert torch.isfinite(a[0]).all()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])


def test_launch_bound_variant_by_occupancy():
    """One loop takes the variant without a register cap; 16 loops in clusters of 16 take the
    capped one, with which all 16 clusters are resident at once."""
    for mode, sfx in ((K.KS_FP64, "f64"), (K.KS_FP32, "f32")):
        with K.KSLoop(22.0, 64, [128], mode) as h:
            assert K.ks_get_option(h.handle, "cluster_min_blocks_" + sfx) == 1
        with K.KSLoop(22.0, 64, [64] * 16, mode) as h:
            assert K.ks_get_option(h.handle, "cluster_" + sfx) == 16
            assert K.ks_get_option(h.handle, "cluster_min_blocks_" + sfx) == 2
            assert K.ks_get_option(h.handle, "cluster_grid_" + sfx) == 256


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
def test_several_loops_per_cluster(mode):
    """More clusters than fit the GPU at once (40 ragged loops in clusters of 16): each cluster
    descends several loops in turn, its mbarriers carrying their phases from one loop to the next
    and the byte counts following each loop's Ns.  Both exchange forms and the per-phase
    launches give the same bits."""
    L, nx = 22.0, 64
    nss = [(32, 64, 128)[i % 3] for i in range(40)]
    u0, T0 = _loops(L, nx, nss, False)
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    outs = []
    for path, xch in ((0, 1), (0, 0), (2, 1)):
        u = torch.tensor(u0, device="cuda").to(dt)
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, chunk=6) as h:
            K.ks_set_option(h.handle, "cluster", 16)
            K.ks_set_option(h.handle, "cluster_exchange", xch)
            K.ks_set_option(h.handle, "path", path)
            if path == 0:
                sfx = "f32" if mode == K.KS_FP32 else "f64"
                assert K.ks_get_option(h.handle, "cluster_" + sfx) == 16
                assert K.ks_get_option(h.handle, "cluster_grid_" + sfx) < 16 * len(nss)
                assert K.ks_get_option(h.handle, "cluster_exchange_" + sfx) == xch
            K.ks_descend(h.handle, u, T, 12, 0.0)
            torch.cuda.synchronize()
        outs.append((u.cpu(), T.cpu()))
    assert torch.isfinite(outs[0][0]).all()
    for o in outs[1:]:
        assert torch.equal(outs[0][0], o[0]) and torch.equal(outs[0][1], o[1])
