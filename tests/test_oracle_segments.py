"""Pins of the oracle's recurrence-loop cut (``oracle.ks_oracle.segment_loop``, Sec. 4.3) and its
norm series, against what the definitions fix: linear interpolation reproduces a trajectory that
is linear in time exactly, returns the saved samples themselves at instants that coincide with
them, starts at the segment's first sample, and the norm of a single Fourier mode is its
closed form."""
import math

import numpy as np
import pytest

from oracle import ks_oracle as ko


def test_linear_in_time_is_exact():
    ts = 0.5 * np.arange(200)
    x = np.linspace(0.0, 1.0, 16, endpoint=False)
    us = 0.3 + 0.7 * ts[:, None] * np.cos(2 * np.pi * x)[None, :] - 0.1 * ts[:, None]
    a, T, Ns = 37, 23.3, 32
    s = ts[a] + T * np.arange(Ns) / Ns
    want = 0.3 + 0.7 * s[:, None] * np.cos(2 * np.pi * x)[None, :] - 0.1 * s[:, None]
    got = ko.segment_loop(ts, us, a, T, Ns)
    assert got.shape == (Ns, 16)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_instants_on_samples_return_the_samples():
    rng = np.random.default_rng(5)
    ts = 0.25 * np.arange(400)
    us = rng.standard_normal((400, 8))
    a, Ns, stride = 11, 16, 3                       # T / Ns = 3 sample intervals
    T = Ns * stride * 0.25
    got = ko.segment_loop(ts, us, a, T, Ns)
    np.testing.assert_array_equal(got, us[a + stride * np.arange(Ns)])
    assert np.array_equal(got[0], us[a])


def test_norm_of_a_single_mode():
    L, nx = 39.0, 64
    x = L * np.arange(nx) / nx
    u = 0.8 * np.sin(2 * np.pi * 3 * x / L)
    assert ko.norm_series(u[None, :], L)[0] == pytest.approx(0.8 * math.sqrt(L / 2), rel=1e-14)

