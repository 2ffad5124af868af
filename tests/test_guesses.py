"""Host logic of the initial-loop pipeline (Sec. 4.3): the recurrence search over a norm series
and the classification of converged loops.  The run, the segment cut and the low-pass run on the
GPU (``test_gpu_dns.py``)."""
import math

import numpy as np
import pytest

from paper_2007_06427_gb300.guesses import recurrence_pairs


def test_recurrence_pairs_on_a_synthetic_norm_series():
    """Maxima of 1 + 0.2 cos(2 pi t / 25) + 0.01 t / 1000 every 25 time units: every pair of
    maxima whose spacing lies in T_range and whose norms differ by less than tol is found, best
    (smallest mismatch) first; maxima before t_min are ignored."""
    ts = 0.5 * np.arange(2000)
    nrm = 1.0 + 0.2 * np.cos(2 * np.pi * ts / 25.0) + 1e-5 * ts
    pairs = recurrence_pairs(ts, nrm, T_range=(20.0, 55.0), tol=1e-3, t_min=100.0)
    assert pairs, "no pairs"
    Ts = [ts[b] - ts[a] for _, a, b in pairs]
    assert set(np.round(Ts, 6)) == {25.0, 50.0}
    assert all(ts[a] >= 100.0 for _, a, _ in pairs)
    mis = [m for m, _, _ in pairs]
    assert mis == sorted(mis)
    for m, a, b in pairs:
        assert m == pytest.approx(abs(nrm[b] - nrm[a]) / nrm[a], rel=1e-15)
        assert m < 1e-3
    # the maxima sit at multiples of 25 (the drift shifts them by less than one sample)
    assert all(abs(ts[a] / 25.0 - round(ts[a] / 25.0)) < 0.05 for _, a, _ in pairs)
    # a tighter tolerance keeps only the spacing-25 pairs (their drift is half as large)
    tight = recurrence_pairs(ts, nrm, T_range=(20.0, 55.0), tol=3.5e-4, t_min=100.0)
    assert tight and all(ts[b] - ts[a] == 25.0 for _, a, b in tight)


def test_recurrence_pairs_respects_the_period_range():
    ts = 0.5 * np.arange(1000)
    nrm = 1.0 + 0.2 * np.cos(2 * np.pi * ts / 10.0)
    pairs = recurrence_pairs(ts, nrm, T_range=(25.0, 35.0), tol=1e-6)
    assert pairs and all(ts[b] - ts[a] == 30.0 for _, a, b in pairs)
    assert recurrence_pairs(ts, nrm, T_range=(11.0, 19.0), tol=1e-6) == []


def test_orbit_classification_closed_forms():
    """u = 0 is trivial, u = a sin(q x) is steady, u = a sin(q x + 2 pi s) has
    ||u_s|| / ||u|| = 2 pi (omega = 2 pi for the first temporal mode)."""
    from paper_2007_06427_gb300.orbits import classify
    L, nx, ns = 39.0, 32, 32
    x = L * np.arange(nx)[None, :] / nx
    s = np.arange(ns)[:, None] / ns
    q = 2 * math.pi * 2 / L
    assert classify(np.zeros((ns, nx)), L)[0] == "trivial"
    kind, norm, ratio = classify(0.7 * np.sin(q * x) + 0 * s, L)
    assert kind == "steady" and ratio < 1e-14 and norm == pytest.approx(0.7 * math.sqrt(L / 2))
    kind, norm, ratio = classify(0.7 * np.sin(q * x + 2 * math.pi * s), L)
    assert kind == "periodic" and ratio == pytest.approx(2 * math.pi, rel=1e-12)
