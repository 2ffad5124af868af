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


def test_converges_to_the_papers_shortest_orbit():
    """Pinned to a number the paper prints: at L = 39 in the centre-symmetric subspace, the stored
    recurrence loop of a chaotic run (T0 = 26.0; ``inputs.orbit_guess``) descends (mixed precision,
    App. C extrapolation, symmetry on) to a periodic orbit of period 25.37, the first of the six
    orbits whose periods Sec. 4.4 lists (to two decimals).  The loop is stored, so the test does
    not depend on a chaotic run, which differs between machines."""
    import json
    import os
    from paper_2007_06427_gb300.inputs import orbit_guess
    from paper_2007_06427_gb300.orbits import Guess, descend_guesses
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                          "paper_setting.json")
    T_paper = json.load(open(golden))["orbit_periods"]["value"][0]
    w = orbit_guess()
    g = Guess(u=w.u[0], T=w.T0[0], t0=w.meta["t0"], mismatch=0.0)
    res = descend_guesses([g], w.L, max_steps=1_500_000, tol=1e-10)
    r = res[0]
    assert r.status == "converged" and r.kind == "periodic", r
    assert r.sqrtJ < 1e-10
    assert abs(r.T - T_paper) < 0.005, (r.T0, r.T)
