"""The orbit-search pipeline end to end on a small case: a centre-symmetric chaotic run,
recurrence loops, their batched mixed-precision descent with the symmetry knob, classification."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ks_oracle as ko
from paper_2007_06427_gb300.orbits import search

pytestmark = pytest.mark.gpu


def test_search_pipeline_small():
    L = 39.0
    gs, res, _, _ = search(L=L, nx=64, ns=32, t_end=1500.0, seed=2, guesses=3,
                           T_range=(10.0, 120.0), rec_tol=0.01, max_steps=30000, tol=1e-10)
    assert len(gs) >= 1 and len(res) == len(gs)
    for g, r in zip(gs, res):
        # the initial sqrt(J) agrees with the oracle's on the projected loop
        ref = ko.residual(g.u, g.T, L, xi=True)
        assert r.sqrtJ0 == pytest.approx(np.sqrt(ref["J"]), rel=1e-10)
        assert r.sqrtJ < r.sqrtJ0
        assert r.status in ("converged", "step_cap", "stalled")
        assert r.kind in ("trivial", "steady", "periodic")
        assert 0 < r.steps <= 30000
