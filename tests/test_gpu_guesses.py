"""The GPU descent started from a recurrence loop of a chaotic run (Sec. 4.3-4.4): J falls
monotonically and by a large factor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.guesses import chaotic_run, recurrence_loops

pytestmark = pytest.mark.gpu


def test_descent_from_recurrence_guess():
    L, nx, ns = 22.0, 32, 32
    ts, us = chaotic_run(L, nx, 2000.0, seed=0)
    g = recurrence_loops(ts, us, L, ns, T_range=(10.0, 80.0), tol=0.005, t_min=200.0,
                         max_loops=1)[0]
    u = torch.tensor(g.u.ravel(), device="cuda")
    T = torch.tensor([g.T], dtype=torch.float64, device="cuda")
    with K.KSLoop(L, nx, [ns], K.KS_FP64, K.KS_IMEX, 0.15, chunk=500) as h:
        J0 = torch.empty(1, dtype=torch.float64, device="cuda")
        K.ks_residual(h.handle, u, T, None, J0)
        sq = torch.zeros(1, dtype=torch.float64, device="cuda")
        K.ks_descend(h.handle, u, T, 20000, 1e-10, None, sq, None)
        hs, hq, _ = K.ks_get_history(h.handle, 0)
    assert np.all(np.diff(hq) <= 0)
    assert sq.item() < 0.05 * np.sqrt(J0.item())
