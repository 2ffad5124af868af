"""The allocation-free residual (ks_residual_noalloc) against the handle-based ks_residual
and against the FP64 CPU oracle.

ks_residual_noalloc serves callers that cannot allocate device memory when they need a
residual (memory pools or arenas that own the device memory, plugins that may not allocate
after start-up, real-time loops).  Its scratch is one file-scope device array shared by all
calls, so this file checks two calls in a row with different sizes (the second call must not
see anything the first left behind) and the rejection of sizes beyond the array's maximum.
It is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ks_oracle as ko
from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop, with_white_noise

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 tolerance of the parity tests


def handle_residual(L, nx, ns, u, T):
    with K.KSLoop(L, nx, [ns], K.KS_FP64) as h:
        r = torch.empty_like(u)
        J = torch.empty(1, dtype=torch.float64, device="cuda")
        K.ks_residual(h.handle, u, torch.tensor([T], dtype=torch.float64, device="cuda"), r, J)
        torch.cuda.synchronize()
    return r.cpu().numpy(), J.item()


def test_noalloc_residual_matches_ks_residual_on_consecutive_calls():
    lib = K.load_library()
    cases = [(22.0, 64, 128, 0), (22.0, 32, 64, 3), (100.0, 256, 256, 1)]
    for L, nx, ns, seed in cases:
        u0, T, _ = spectral_loop(seed, nx, L, ns=ns, T_range=(20.0, 80.0),
                                 decay=(max(2.0, (nx // 3) / 10.0), 2.0))
        u = torch.from_numpy(u0.ravel()).cuda()
        r = torch.full_like(u, float("nan"))
        J = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.ks_residual_noalloc(L, nx, ns, u.data_ptr(), T, r.data_ptr(), J.data_ptr(), None)
        assert rc == K.KS_OK, K.ks_last_error()
        torch.cuda.synchronize()
        r_ref, J_ref = handle_residual(L, nx, ns, u, T)
        rn = r.cpu().numpy()
        assert np.linalg.norm(rn - r_ref) <= TOL * np.linalg.norm(r_ref)
        assert abs(J.item() - J_ref) <= TOL * J_ref


def test_noalloc_rejects_sizes_beyond_its_array():
    lib = K.load_library()
    u = torch.zeros(512 * 64, dtype=torch.float64, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.ks_residual_noalloc(22.0, 512, 64, u.data_ptr(), 40.0, None, J.data_ptr(), None)
    assert rc == K.KS_ERR_ARG
    assert "256" in K.ks_last_error()
    rc = lib.ks_residual_noalloc(22.0, 64, 512, u.data_ptr(), 40.0, None, J.data_ptr(), None)
    assert rc == K.KS_ERR_ARG
    host = np.zeros(64 * 64)
    rc = lib.ks_residual_noalloc(22.0, 64, 64, host.ctypes.data, 40.0, None, J.data_ptr(), None)
    assert rc == K.KS_ERR_ARG


def test_noalloc_residual_matches_oracle():
    """r and J straight against the oracle, element by element (norm and worst element), on a
    band-limited loop and on one carrying white noise in every grid mode (the projection onto
    the band is part of the call)."""
    lib = K.load_library()
    for L, nx, ns, seed, noise in [(22.0, 64, 128, 0, 0.0), (22.0, 64, 128, 0, 0.5),
                                   (22.0, 16, 256, 2, 0.5)]:
        u0, T, _ = spectral_loop(seed, nx, L, ns=ns, T_range=(20.0, 80.0))
        if noise:
            u0 = with_white_noise(u0, seed, noise)
        u = torch.from_numpy(u0.ravel()).cuda()
        r = torch.full_like(u, float("nan"))
        J = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.ks_residual_noalloc(L, nx, ns, u.data_ptr(), T, r.data_ptr(), J.data_ptr(), None)
        assert rc == K.KS_OK, K.ks_last_error()
        torch.cuda.synchronize()
        ref = ko.residual(u0, T, L)
        rn = r.cpu().numpy().reshape(ns, nx)
        assert np.linalg.norm(rn - ref["r"]) <= TOL * np.linalg.norm(ref["r"])
        assert np.abs(rn - ref["r"]).max() <= TOL * np.abs(ref["r"]).max()
        assert abs(J.item() - ref["J"]) <= TOL * ref["J"]


def test_noalloc_rejects_bad_period():
    lib = K.load_library()
    u = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for T in (0.0, -1.0, float("nan"), float("inf")):
        rc = lib.ks_residual_noalloc(22.0, 64, 64, u.data_ptr(), T, None, J.data_ptr(), None)
        assert rc == K.KS_ERR_ARG, T
        assert "T" in K.ks_last_error()
