"""J(u, T) as an autograd Function with the hand-written adjoint backward: gradcheck against
centred finite differences (h = 1e-6) and the oracle's gradient, batch of 16 loops of 64 x 64
at L = 22 in FP64, plus the FP32 handle against the oracle at 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ks_oracle as ko
from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.autograd import cost
from paper_2007_06427_gb300.inputs import workload, spectral_loop

pytestmark = pytest.mark.gpu


def test_gradcheck_tiny_full():
    """Full Jacobian check on a tiny ragged batch (every grid value and T)."""
    L, nx, nss = 22.0, 8, [8, 16]
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i, nx, L, ns=n, T_range=(20.0, 80.0))
        us.append(u)
        Ts.append(T)
    u = torch.tensor(np.concatenate([a.ravel() for a in us]), device="cuda", requires_grad=True)
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda", requires_grad=True)
    with K.KSLoop(L, nx, nss, K.KS_FP64) as h:
        assert torch.autograd.gradcheck(lambda a, b: cost(a, b, h), (u, T), eps=1e-6,
                                        atol=1e-6, rtol=1e-5)


def test_gradcheck_batch16_64x64_fp64():
    w = workload("batch16_64x64")
    u = torch.tensor(w.packed(), device="cuda", requires_grad=True)
    T = torch.tensor(w.T0, dtype=torch.float64, device="cuda", requires_grad=True)
    with K.KSLoop(w.L, w.nx, w.ns, K.KS_FP64) as h:
        assert torch.autograd.gradcheck(lambda a, b: cost(a, b, h), (u, T), eps=1e-6,
                                        atol=1e-5, rtol=1e-5, fast_mode=True)
        J = cost(u, T, h)
        J.sum().backward()
    gu = u.grad.cpu().numpy()
    off = 0
    for b in range(w.batch):
        n = w.ns[b]
        ref = ko.adjoint_grad(w.u[b], w.T0[b], w.L)
        exact = 2 * w.L / (w.nx * n) * ref["G"].ravel()
        got = gu[off:off + n * w.nx]
        off += n * w.nx
        assert np.linalg.norm(got - exact) <= 1e-12 * np.linalg.norm(exact)
        assert abs(T.grad[b].item() - ref["dJdT"]) <= 1e-12 * abs(ref["dJdT"])
        assert abs(J[b].item() - ref["J"]) <= 1e-12 * ref["J"]


def test_batch16_64x64_fp32_gradient():
    w = workload("batch16_64x64")
    w.u = [a.astype(np.float32).astype(np.float64) for a in w.u]   # the handle's float input
    u = torch.tensor(w.packed(), dtype=torch.float32, device="cuda", requires_grad=True)
    T = torch.tensor(w.T0, dtype=torch.float64, device="cuda", requires_grad=True)
    with K.KSLoop(w.L, w.nx, w.ns, K.KS_FP32) as h:
        J = cost(u, T, h)
        (J * torch.arange(1, w.batch + 1, device="cuda")).sum().backward()
    gu = u.grad.double().cpu().numpy()
    off = 0
    for b in range(w.batch):
        n = w.ns[b]
        ref = ko.adjoint_grad(w.u[b], w.T0[b], w.L)
        exact = (b + 1) * 2 * w.L / (w.nx * n) * ref["G"].ravel()
        got = gu[off:off + n * w.nx]
        off += n * w.nx
        assert np.linalg.norm(got - exact) <= 1e-5 * np.linalg.norm(exact)
        assert abs(T.grad[b].item() - (b + 1) * ref["dJdT"]) <= 1e-5 * abs((b + 1) * ref["dJdT"])


def test_gradcheck_in_centre_symmetric_subspace():
    """With the "symmetry" knob the cost is J(P_Xi P u) and its gradient the projected G:
    full Jacobian check on a tiny ragged batch from non-invariant inputs."""
    L, nx, nss = 22.0, 8, [8, 16]
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i + 3, nx, L, ns=n, T_range=(20.0, 80.0))
        us.append(u)
        Ts.append(T)
    u = torch.tensor(np.concatenate([a.ravel() for a in us]), device="cuda", requires_grad=True)
    T = torch.tensor(Ts, dtype=torch.float64, device="cuda", requires_grad=True)
    with K.KSLoop(L, nx, nss, K.KS_FP64) as h:
        K.ks_set_option(h.handle, "symmetry", 1)
        assert torch.autograd.gradcheck(lambda a, b: cost(a, b, h), (u, T), eps=1e-6,
                                        atol=1e-6, rtol=1e-5)
        J = cost(u, T, h)
    for b in range(len(nss)):
        assert abs(J[b].item() - ko.residual(us[b], Ts[b], L, xi=True)["J"]) <= 1e-12 * J[b].item()
