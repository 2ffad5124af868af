"""The host-side extrapolated descent (accel._core, App. C as read) on a stand-in for the library
(no GPU): a linear contraction toward a fixed point l* = (u*, T*), one step multiplying the
distance by rho.  The geometric extrapolation is exact for it, so the first move lands on l*;
with two decay rates it is not, and each move is kept only when it lowers sqrt(J)."""
import math
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import accel


class FakeLib(types.SimpleNamespace):
    """Steps act on the resident state: u <- u* + D (u - u*), T <- T* + d (T - T*)."""

    KS_RUNNING, KS_CONVERGED, KS_STEP_CAP = 0, 1, 2

    def __init__(self, ustar, Tstar, rates, rateT):
        super().__init__()
        self.ustar, self.Tstar = ustar, Tstar
        self.rates, self.rateT = rates, rateT
        self.u = None
        self.T = None
        self.steps = 0

    def ks_set_state(self, h, u, T):
        self.u, self.T, self.steps = u.clone(), T.clone(), 0

    def ks_step(self, h, n, tol):
        for _ in range(n):
            self.u = self.ustar + self.rates * (self.u - self.ustar)
            self.T = self.Tstar + self.rateT * (self.T - self.Tstar)
        self.steps += n

    def ks_get_state(self, h, u, T, steps, sq, st):
        u.copy_(self.u)
        T.copy_(self.T)
        steps.fill_(self.steps)
        st.fill_(self.KS_RUNNING)


def run(fake, u0, T0, **kw):
    accel.K, saved = fake, accel.K
    try:
        fake.ks_set_state(None, u0, T0)
        sqrtJ = lambda u, T: float(torch.linalg.norm(u - fake.ustar))  # noqa: E731
        hist = []
        out = accel._core(None, u0.clone(), T0.clone(), sqrtJ, kw.get("tol", 1e-12),
                          kw.get("max_steps", 20000), kw.get("start", 1.0), kw.get("drop", 0.5),
                          kw.get("chunk", 50), 0, hist)
    finally:
        accel.K = saved
    return out, hist


def test_one_move_lands_on_the_fixed_point_of_a_single_rate():
    ustar = torch.tensor([0.3, -1.2, 2.0], dtype=torch.float64)
    rho = 0.98
    fake = FakeLib(ustar, torch.tensor([40.0], dtype=torch.float64),
                   torch.full((3,), rho, dtype=torch.float64), rho)
    u0 = ustar + torch.tensor([1.0, 0.5, -0.25], dtype=torch.float64)
    (u, T, sq, total, status, nex, nrej, _), hist = run(fake, u0, torch.tensor([41.0], dtype=torch.float64))
    assert status == fake.KS_CONVERGED and nex == 1 and nrej == 0
    assert torch.allclose(u, ustar, rtol=0, atol=1e-12) and abs(T.item() - 40.0) < 1e-12
    # anchor after the first chunk, move after the second (rho^50 = 0.36 < 1/2), then converged
    assert total == 100


def test_two_rates_need_several_moves_and_sqrtJ_never_rises():
    ustar = torch.zeros(2, dtype=torch.float64)
    fake = FakeLib(ustar, torch.tensor([40.0], dtype=torch.float64),
                   torch.tensor([0.99, 0.9], dtype=torch.float64), 0.99)
    u0 = torch.tensor([1.0, 1.0], dtype=torch.float64)
    (u, T, sq, total, status, nex, nrej, _), hist = run(fake, u0, torch.tensor([41.0], dtype=torch.float64),
                                                     tol=1e-10)
    assert status == fake.KS_CONVERGED and sq < 1e-10 and nex >= 1
    plain_steps = math.ceil(math.log(1e-10) / math.log(0.99))
    assert total < plain_steps / 2
    kept = [s for _, s, ev in hist if ev != "rejected"]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(kept, kept[1:]))
