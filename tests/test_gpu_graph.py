"""The graph-captured four-launch form (path 2, knob "graph") against the same launches issued one
by one: bit-identical states, the same number of kernel launches, and replays that happen.

Runs of up to 16 tau-steps are captured as CUDA graphs and replayed; an odd last step is launched
directly.  37 steps exercise a full 16-step graph (twice), a 4-step graph and one direct step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu


def loops(nx, nss, L=22.0, T_range=(20.0, 80.0), scale=None):
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i, nx, L, ns=n, T_range=T_range, decay=(2.0, 2.0))
        us.append(u * (scale[i] if scale else 1.0))
        Ts.append(T)
    return us, Ts


def to_dev(us, Ts, mode):
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).to("cuda", dt)
    return u, torch.tensor(Ts, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("symmetry", [0, 1])
@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
def test_graph_steps_equal_direct_launches(mode, symmetry):
    L, nx, nss = 22.0, 64, [32, 64, 128, 256, 64, 32]
    us, Ts = loops(nx, nss, L)
    out = {}
    for graph in (0, 1):
        u, T = to_dev(us, Ts, mode)
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15) as h:
            K.ks_set_option(h.handle, "path", 2)
            K.ks_set_option(h.handle, "symmetry", symmetry)
            K.ks_set_option(h.handle, "graph", graph)
            assert K.ks_get_option(h.handle, "graph") == graph
            K.ks_set_state(h.handle, u, T)
            K.ks_profile_read(h.handle, reset=True)
            K.ks_step(h.handle, 37, 0.0)
            K.ks_step(h.handle, 5, 0.0)          # cached graphs of the other parity / length
            _, launches = K.ks_profile_read(h.handle)
            replays = K.ks_get_option(h.handle, "graph_replays")
            K.ks_get_state(h.handle, u, T)
            torch.cuda.synchronize()
        out[graph] = (u.cpu(), T.cpu(), launches, replays)
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] >= 42 * 4   # (plus the priming transform of the state)
    assert out[0][3] == 0
    assert out[1][3] == 2 + 1 + 1          # 16, 16, 4 | 4


def test_graph_mixed_batch_in_both_precisions_equals_direct():
    """A mixed batch whose loops switch to double at different times: while both precisions
    are live, each captured step holds the float and double chains as parallel branches."""
    L, nx, nss = 22.0, 32, [32, 32, 64, 32]
    us, Ts = loops(nx, nss, L, T_range=(30.0, 50.0), scale=(1e-2, 3e-3, 1e-2, 1.0))
    outs = []
    for graph in (0, 1):
        u, T = to_dev(us, Ts, K.KS_FP64)
        steps = torch.zeros(4, dtype=torch.int64, device="cuda")
        sq = torch.zeros(4, dtype=torch.float64, device="cuda")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        with K.KSLoop(L, nx, nss, K.KS_MIXED, K.KS_IMEX, 0.15, tol=1e-10, switch_tol=1e-5,
                      chunk=500) as h:
            K.ks_set_option(h.handle, "path", 2)
            K.ks_set_option(h.handle, "graph", graph)
            K.ks_descend(h.handle, u, T, 60000, 1e-10, steps, sq, st)
            hp = [K.ks_get_history(h.handle, b)[2] for b in range(4)]
            replays = K.ks_get_option(h.handle, "graph_replays")
        outs.append((u.cpu(), T.cpu(), steps.cpu(), st.cpu()))
        assert any((hp[a][i] == 1) and (hp[b][i] == 0)
                   for a in range(4) for b in range(4)
                   for i in range(min(len(hp[a]), len(hp[b]))))
        assert (replays > 0) == bool(graph)
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("forms", [(0, 2), (2, 0), (1, 2), (2, 1), (2, 2)])
def test_per_precision_launch_forms_equal_cluster_forms(forms):
    """Each precision of a mixed batch stepped by its own launch form (float form, double form):
    the descent through the switch, with loops live in both precisions at once, equals the one
    with both precisions in the cluster-resident form bit for bit."""
    L, nx, nss = 22.0, 32, [32, 32, 64, 32]
    us, Ts = loops(nx, nss, L, T_range=(30.0, 50.0), scale=(1e-2, 3e-3, 1e-2, 1.0))
    outs = []
    for f32, f64 in ((0, 0), forms):
        u, T = to_dev(us, Ts, K.KS_FP64)
        steps = torch.zeros(4, dtype=torch.int64, device="cuda")
        sq = torch.zeros(4, dtype=torch.float64, device="cuda")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        with K.KSLoop(L, nx, nss, K.KS_MIXED, K.KS_IMEX, 0.15, tol=1e-10, switch_tol=1e-5,
                      chunk=500) as h:
            K.ks_set_option(h.handle, "finish_f32_adjoint", 0)
            K.ks_set_option(h.handle, "path_f32", f32)
            K.ks_set_option(h.handle, "path_f64", f64)
            K.ks_descend(h.handle, u, T, 60000, 1e-10, steps, sq, st)
        outs.append((u.cpu(), T.cpu(), steps.cpu(), st.cpu()))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("symmetry", [0, 1])
@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32])
def test_item_block_sizes_give_the_same_bits(mode, symmetry):
    """Row and column items of 256 threads (knobs "row_threads", "col_threads"): the column
    partials of J and L^dag_2 keep their 128 accumulators, so the descent and the reported
    sqrt(J) equal those of 128-thread items bit for bit."""
    L, nx, nss = 22.0, 64, [32, 64, 128, 256, 64, 32]
    us, Ts = loops(nx, nss, L)
    out = []
    for rt, ct in ((128, 128), (256, 128), (128, 256), (256, 256)):
        u, T = to_dev(us, Ts, mode)
        sq = torch.zeros(len(nss), dtype=torch.float64, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15) as h:
            K.ks_set_option(h.handle, "path", 2)
            K.ks_set_option(h.handle, "symmetry", symmetry)
            K.ks_set_option(h.handle, "row_threads", rt)
            K.ks_set_option(h.handle, "col_threads", ct)
            assert (K.ks_get_option(h.handle, "row_threads"), K.ks_get_option(h.handle, "col_threads")) == (rt, ct)
            K.ks_set_state(h.handle, u, T)
            K.ks_step(h.handle, 9, 0.0)
            K.ks_get_state(h.handle, u, T, None, sq)
            torch.cuda.synchronize()
        out.append((u.cpu(), T.cpu(), sq.cpu()))
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert torch.equal(a, b)
