"""Checkpoint / resume: a descent interrupted and resumed from an .npz checkpoint continues
bit for bit; a corrupt checkpoint is rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import checkpoint
from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu


def _state(mode, nx, nss, L=22.0):
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i, nx, L, ns=n, T_range=(20.0, 80.0))
        us.append(u)
        Ts.append(T)
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    u = torch.tensor(np.concatenate([a.ravel() for a in us]), device="cuda").to(dt)
    return u, torch.tensor(Ts, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32, K.KS_MIXED])
def test_resume_is_bitwise(mode, tmp_path):
    L, nx, nss = 22.0, 32, [32, 64]
    u, T = _state(mode, nx, nss, L)
    sw = 10.0 if mode == K.KS_MIXED else 0.0      # mixed: switch one loop early
    # reference with the same call boundaries (a mixed handle hands switched loops to double
    # at the end of a call, so 10 + 10 steps is not 20 steps once a loop switches)
    with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, switch_tol=sw) as h:
        K.ks_set_state(h.handle, u, T)
        K.ks_step(h.handle, 10, 0.0)
        K.ks_step(h.handle, 10, 0.0)
        ref_u, ref_T = torch.empty_like(u), torch.empty_like(T)
        ref_steps = torch.zeros(2, dtype=torch.int64, device="cuda")
        K.ks_get_state(h.handle, ref_u, ref_T, ref_steps)
    with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, switch_tol=sw) as h:
        K.ks_set_state(h.handle, u, T)
        K.ks_step(h.handle, 10, 0.0)
        checkpoint.save(h, str(tmp_path / "ck.npz"), switch_tol=sw)
    h2 = checkpoint.resume(str(tmp_path / "ck.npz"))
    try:
        K.ks_step(h2.handle, 10, 0.0)
        u2, T2 = torch.empty_like(u), torch.empty_like(T)
        st2 = torch.zeros(2, dtype=torch.int64, device="cuda")
        K.ks_get_state(h2.handle, u2, T2, st2)
    finally:
        h2.close()
    assert torch.equal(u2, ref_u) and torch.equal(T2, ref_T)
    assert st2.tolist() == ref_steps.tolist()
    if mode != K.KS_MIXED:
        assert st2.tolist() == [20, 20]


def test_corrupt_checkpoint_rejected(tmp_path):
    L, nx, nss = 22.0, 32, [32]
    u, T = _state(K.KS_FP64, nx, nss, L)
    with K.KSLoop(L, nx, nss, K.KS_FP64) as h:
        K.ks_set_state(h.handle, u, T)
        checkpoint.save(h, str(tmp_path / "ck.npz"))
    z = dict(np.load(tmp_path / "ck.npz"))
    z["band"] = z["band"][:-2]
    np.savez(tmp_path / "bad.npz", **z)
    with pytest.raises(ValueError):
        checkpoint.resume(str(tmp_path / "bad.npz"))
    del z["T"]
    np.savez(tmp_path / "bad2.npz", **z)
    with pytest.raises(ValueError):
        checkpoint.resume(str(tmp_path / "bad2.npz"))


def test_knobs_status_and_history_travel_with_the_checkpoint(tmp_path):
    """The descent knobs are restored on resume; statuses and histories come back to the caller
    as saved (a loop that converged before the checkpoint freezes again before its next step)."""
    L, nx, nss = 22.0, 32, [32, 32]
    u, T = _state(K.KS_FP64, nx, nss, L)
    u[: 32 * nx] = 0.0                              # loop 0: u = 0, converged at once
    knobs = {"symmetry": 1, "extrapolate": 1, "extrapolate_start_ppm": 2000,
             "extrapolate_drop_ppm": 400000, "stall_window": 12345, "stall_drop_ppm": 77,
             "chunk": 50}
    with K.KSLoop(L, nx, nss, K.KS_FP64, K.KS_IMEX, 0.15) as h:
        for k, v in knobs.items():
            K.ks_set_option(h.handle, k, v)
        K.ks_descend(h.handle, u, T, 100, 1e-10)
        checkpoint.save(h, str(tmp_path / "ck.npz"))
        hs0, hq0, _ = K.ks_get_history(h.handle, 1)
    h2, saved = checkpoint.resume(str(tmp_path / "ck.npz"), info=True)
    try:
        for k, v in knobs.items():
            assert K.ks_get_option(h2.handle, k) == v, k
        assert saved["status"] == [K.KS_CONVERGED, K.KS_STEP_CAP]
        np.testing.assert_array_equal(saved["history"][1][0], hs0)
        np.testing.assert_array_equal(saved["history"][1][1], hq0)
        steps = torch.zeros(2, dtype=torch.int64, device="cuda")
        st = torch.zeros(2, dtype=torch.int32, device="cuda")
        K.ks_step(h2.handle, 5, 1e-10)
        K.ks_get_state(h2.handle, None, None, steps, None, st)
        assert steps.tolist() == [0, 105] and st.tolist()[0] == K.KS_CONVERGED
    finally:
        h2.close()
