"""Failure detection without faulting the GPU: a bounded barrier wait that runs out, per-loop
freeze on divergence, the no-progress (stall) test, and argument errors on a live handle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu


def loops(nx, nss, L=22.0):
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i, nx, L, ns=n, T_range=(20.0, 80.0))
        us.append(u)
        Ts.append(T)
    u = torch.tensor(np.concatenate([a.ravel() for a in us]), device="cuda")
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda")
    return u, T


def test_grid_barrier_wait_runs_out_and_reports_timeout():
    """The grid-persistent kernel's barrier waits for one arrival that never comes: every
    wait gives up after about a second, the kernel returns, and the read-back reports
    KS_ERR_TIMEOUT.  The handle then works again."""
    u, T = loops(32, [32, 64])
    with K.KSLoop(22.0, 32, [32, 64], K.KS_FP64, chunk=4) as h:
        K.ks_set_option(h.handle, "path", 1)
        K.ks_set_option(h.handle, "test_barrier_timeout", 1)
        with pytest.raises(K.KsError) as e:
            K.ks_descend(h.handle, u.clone(), T.clone(), 4, 0.0)
        assert e.value.code == K.KS_ERR_TIMEOUT
        K.ks_set_option(h.handle, "test_barrier_timeout", 0)
        u2, T2 = u.clone(), T.clone()
        st = torch.zeros(2, dtype=torch.int32, device="cuda")
        K.ks_descend(h.handle, u2, T2, 4, 0.0, None, None, st)
        assert st.tolist() == [K.KS_STEP_CAP] * 2
        ref_u, ref_T = u.clone(), T.clone()
        K.ks_set_option(h.handle, "path", 2)
        K.ks_descend(h.handle, ref_u, ref_T, 4, 0.0)
        assert torch.equal(u2, ref_u) and torch.equal(T2, ref_T)


def test_stall_detection_marks_loops_stalled():
    """A no-progress window that no descent can satisfy ends a double descent as STALLED."""
    u, T = loops(32, [32, 32])
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    steps = torch.zeros(2, dtype=torch.int64, device="cuda")
    with K.KSLoop(22.0, 32, [32, 32], K.KS_FP64, chunk=10) as h:
        K.ks_set_option(h.handle, "stall_window", 10)
        K.ks_set_option(h.handle, "stall_drop_ppm", 999999)
        K.ks_descend(h.handle, u, T, 1000, 0.0, steps, None, st)
    assert st.tolist() == [K.KS_STALLED] * 2
    assert steps.tolist() == [20, 20]


def test_mixed_stall_switches_to_double_first():
    """In a mixed descent the same test first hands the loop to double, then stalls it."""
    u, T = loops(32, [32])
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    with K.KSLoop(22.0, 32, [32], K.KS_MIXED, chunk=10) as h:
        K.ks_set_option(h.handle, "stall_window", 10)
        K.ks_set_option(h.handle, "stall_drop_ppm", 999999)
        K.ks_descend(h.handle, u, T, 1000, 0.0, steps, None, st)
        hs, hq, hp = K.ks_get_history(h.handle, 0)
    assert st.tolist() == [K.KS_STALLED]
    assert 1 in hp.tolist() and 0 in hp.tolist()


def test_bad_calls_on_a_live_handle():
    u, T = loops(32, [32])
    with K.KSLoop(22.0, 32, [32], K.KS_FP64) as h:
        with pytest.raises(K.KsError) as e:
            K.ks_step(h.handle, 1)
        assert e.value.code == K.KS_ERR_STATE
        with pytest.raises(K.KsError) as e:
            K.ks_residual(h.handle, None, T)
        assert e.value.code == K.KS_ERR_ARG
        with pytest.raises(K.KsError) as e:
            K.ks_set_option(h.handle, "no_such_knob", 1)
        assert e.value.code == K.KS_ERR_ARG
        with pytest.raises(K.KsError) as e:
            K.ks_set_option(h.handle, "cluster", 17)
        assert e.value.code == K.KS_ERR_ARG
