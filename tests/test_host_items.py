"""The per-CTA work items of the per-phase launches (ks_items.cuh), compiled as sequential host
code (KS_HOST_EMULATION) by tests/host/ks_host_step.cpp, against the oracle: analysis of a grid
loop onto its band, tau-steps through the four phases or the residual and adjoint gradient,
synthesis back to the grid; in double and in float, plain and in the centre-symmetric subspace.  No GPU: this
pins the items' index arithmetic and formulas on the CPU.  The GPU tests check that the cluster
and persistent kernels reproduce these items bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2007_06427_gb300 import build as B
from paper_2007_06427_gb300.inputs import spectral_loop

HERE = os.path.dirname(os.path.abspath(__file__))


_EXE = {}


def harness_exe():
    return _EXE["path"]


@pytest.fixture(scope="module", autouse=True)
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("items") / "ks_host_step"
    subprocess.run([cxx, "-std=c++17", "-O1", "-w", "-I", B.CSRC,
                    os.path.join(HERE, "host", "ks_host_step.cpp"), "-o", str(exe)], check=True)
    _EXE["path"] = str(exe)
    return str(exe)


def run_batch(exe, loops, L, dtau, scheme, steps, mode=0, prec=64, xi=0, tol=0.0, status=False,
              switch_tol=0.0):
    """loops: [(u[n][m], T)]; returns [(a, c, grid)] per loop (mode 0: sqrt(J0), T after the
    steps, u; modes 1 and 2: J, dJ/dT, and G or r), and with status=True also the loops'
    (status, steps taken)."""
    nx = loops[0][0].shape[1]
    inp = f"{L!r} {nx} {len(loops)} {dtau!r} {scheme} {steps} {mode} {prec} {xi} {tol!r} {switch_tol!r}\n"
    inp += "\n".join(f"{u.shape[0]} {float(T)!r}" for u, T in loops) + "\n"
    inp += "\n".join(repr(float(x)) for u, _ in loops for x in u.ravel())
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    res, st, o = [], [], 4 * len(loops)
    for b, (u, _) in enumerate(loops):
        n = u.size
        res.append((float(out[4 * b]), float(out[4 * b + 1]),
                    np.array(list(map(float, out[o:o + n]))).reshape(u.shape)))
        st.append((int(out[4 * b + 2]), int(out[4 * b + 3])))
        o += n
    return (res, st) if status else res


def run(exe, u, T, L, dtau, scheme, steps, mode=0, prec=64, xi=0):
    return run_batch(exe, [(u, T)], L, dtau, scheme, steps, mode, prec, xi)[0]


@pytest.mark.parametrize("nx,ns,L,scheme,dtau,steps", [
    (32, 32, 22.0, ko.IMEX, 0.15, 5),
    (32, 64, 22.0, ko.IMEX, 0.15, 3),
    (64, 32, 39.0, ko.IMEX, 0.15, 4),
    (16, 16, 22.0, ko.EXPLICIT, 1e-3, 3),
    (8, 8, 22.0, ko.IMEX, 0.15, 2),
    (16, 128, 22.0, ko.IMEX, 0.15, 2),
    (16, 16, 22.0, ko.IMEX, 0.15, 200),       # a trajectory: rounding does not grow
])
def test_items_step_matches_oracle(harness, nx, ns, L, scheme, dtau, steps):
    u, T, _ = spectral_loop(1, nx, L, ns=ns, T_range=(30.0, 50.0))
    sq0, Tn, g = run(harness, u, T, L, dtau, scheme, steps)
    ref = ko.descend(u, T, L, dtau, scheme, steps)
    J0 = ko.residual(u, T, L)["J"]
    assert abs(sq0 - np.sqrt(J0)) <= 1e-12 * np.sqrt(J0)
    assert np.linalg.norm(g - ref["u"]) <= 1e-12 * np.linalg.norm(ref["u"])
    assert abs(Tn - ref["T"]) <= 1e-12 * abs(ref["T"])
    assert ref["T"] != T and np.linalg.norm(ref["u"] - u) > 1e-6 * np.linalg.norm(u)


def test_items_analysis_synthesis_is_the_band_projection(harness):
    """Zero steps: analysis then synthesis returns the band-limited part of the loop."""
    u, T, _ = spectral_loop(2, 32, 22.0, ns=64, T_range=(30.0, 50.0))
    noise = np.random.default_rng(0).standard_normal(u.shape)   # energy outside the band too
    v = u + 0.1 * noise
    _, Tn, g = run(harness, v, T, 22.0, 0.15, ko.IMEX, 0)
    ref = ko.descend(v, T, 22.0, 0.15, ko.IMEX, 0)["u"]
    assert Tn == T
    assert np.linalg.norm(g - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(g - v) > 1e-3 * np.linalg.norm(v)


SHAPES = [(32, 32, 22.0), (32, 64, 22.0), (64, 32, 39.0), (16, 128, 22.0)]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("nx,ns,L", SHAPES)
@pytest.mark.parametrize("xi", [0, 1])
def test_items_gradient_matches_oracle_fp64(harness, nx, ns, L, xi):
    """r, J, G = L^dag_1 r and dJ/dT (Eq. KS_R, Eq. KS_L_dagger) within 1e-12."""
    u, T, _ = spectral_loop(1, nx, L, ns=ns, T_range=(30.0, 50.0), symmetric=bool(xi))
    J, dJdT, G = run(harness, u, T, L, 0.15, ko.IMEX, 0, mode=1, prec=64, xi=xi)
    ref = ko.adjoint_grad(u, T, L, xi=bool(xi))
    assert rel(G, ref["G"]) <= 1e-12
    _, _, r = run(harness, u, T, L, 0.15, ko.IMEX, 0, mode=2, prec=64, xi=xi)
    assert rel(r, ko.residual(u, T, L, xi=bool(xi))["r"]) <= 1e-12
    assert abs(J - ref["J"]) <= 1e-12 * ref["J"]
    assert abs(dJdT - ref["dJdT"]) <= 1e-12 * abs(ref["dJdT"])


@pytest.mark.parametrize("nx,ns,L", SHAPES)
@pytest.mark.parametrize("xi", [0, 1])
def test_items_float_path_matches_oracle(harness, nx, ns, L, xi):
    """The float items (float-float partials for J and L^dag_2) within 1e-5 of the oracle given
    the same float-rounded field: gradient, and three IMEX steps."""
    u, T, _ = spectral_loop(1, nx, L, ns=ns, T_range=(30.0, 50.0), symmetric=bool(xi))
    uf = u.astype(np.float32).astype(np.float64)
    J, dJdT, G = run(harness, uf, T, L, 0.15, ko.IMEX, 0, mode=1, prec=32, xi=xi)
    ref = ko.adjoint_grad(uf, T, L, xi=bool(xi))
    assert rel(G, ref["G"]) <= 1e-5
    assert abs(J - ref["J"]) <= 1e-5 * ref["J"]
    assert abs(dJdT - ref["dJdT"]) <= 1e-5 * abs(ref["dJdT"])
    _, Tn, g = run(harness, uf, T, L, 0.15, ko.IMEX, 3, mode=0, prec=32, xi=xi)
    d = ko.descend(uf, T, L, 0.15, ko.IMEX, 3, xi=bool(xi))
    assert rel(g, d["u"]) <= 1e-5 and abs(Tn - d["T"]) <= 1e-5 * d["T"]


def test_items_symmetric_step_keeps_the_loop_odd(harness):
    """With the symmetry knob a centre-symmetric loop stays odd in x after steps."""
    u, T, _ = spectral_loop(3, 32, 22.0, ns=32, T_range=(30.0, 50.0), symmetric=True)
    _, _, g = run(harness, u, T, 22.0, 0.15, ko.IMEX, 4, mode=0, prec=64, xi=1)
    reflected = -np.roll(g[:, ::-1], 1, axis=1)      # u(-x) on the grid m -> -m mod Nx
    assert np.abs(g - reflected).max() <= 1e-13 * np.abs(g).max()


@pytest.mark.parametrize("mode", [0, 1])
def test_items_ragged_batch_matches_oracle(harness, mode):
    """A ragged batch (Ns 8 .. 128, columns longest loop first, per-loop offsets): every loop
    agrees with the oracle run on it alone."""
    L, nx = 22.0, 32
    loops = []
    for i, n in enumerate([32, 8, 128, 16, 64, 32]):
        u, T, _ = spectral_loop(10 + i, nx, L, ns=n, T_range=(30.0, 50.0))
        loops.append((u, T))
    res = run_batch(harness, loops, L, 0.15, ko.IMEX, 3, mode=mode)
    for (u, T), (a, c, g) in zip(loops, res):
        if mode == 0:
            ref = ko.descend(u, T, L, 0.15, ko.IMEX, 3)
            assert rel(g, ref["u"]) <= 1e-12 and abs(c - ref["T"]) <= 1e-12 * ref["T"]
            assert abs(a - np.sqrt(ko.residual(u, T, L)["J"])) <= 1e-12 * a
        else:
            ref = ko.adjoint_grad(u, T, L)
            assert rel(g, ref["G"]) <= 1e-12 and abs(a - ref["J"]) <= 1e-12 * ref["J"]
            assert abs(c - ref["dJdT"]) <= 1e-12 * abs(ref["dJdT"])


def test_items_freeze_rules():
    """The per-loop freeze of the update item (convergence test of Sec. 4.3, divergence): a
    converged loop stops before the step whose starting sqrt(J) is below tol and keeps its T; a
    non-finite loop is frozen as diverged; the other loops of the batch run on."""
    L, nx = 22.0, 16
    u0, T0, _ = spectral_loop(4, nx, L, ns=16, T_range=(30.0, 50.0))
    u1, T1, _ = spectral_loop(5, nx, L, ns=16, T_range=(30.0, 50.0))
    flat = np.full((16, nx), 0.25)                    # u = const: r = 0 (an equilibrium)
    bad = u1.copy()
    bad[3, 5] = np.nan
    loops = [(u0, T0), (flat, 35.0), (bad, T1)]
    (res, st) = run_batch(harness_exe(), loops, L, 0.15, ko.IMEX, 4, tol=1e-10, status=True)
    assert st[0] == (0, 4)                           # running, all four steps taken
    assert st[1][0] == 1 and st[1][1] == 0 and res[1][1] == 35.0   # converged at once, T kept
    assert st[2][0] == 4 and st[2][1] == 0           # diverged, no step taken
    ref = ko.descend(u0, T0, L, 0.15, ko.IMEX, 4)
    assert rel(res[0][2], ref["u"]) <= 1e-12


def test_items_float_switch_rule():
    """The float update item hands a loop to the double phase (status switch, no step taken)
    once its sqrt(J) is at or below switch_tol; a loop above it steps on."""
    L, nx = 22.0, 16
    small, T0, _ = spectral_loop(6, nx, L, ns=16, T_range=(30.0, 50.0))
    big, T1, _ = spectral_loop(7, nx, L, ns=16, T_range=(30.0, 50.0))
    small = 1e-4 * small
    sq_small = np.sqrt(ko.residual(small, T0, L)["J"])
    sq_big = np.sqrt(ko.residual(big, T1, L)["J"])
    sw = 10 * sq_small
    assert sw < sq_big
    res, st = run_batch(harness_exe(), [(small, T0), (big, T1)], L, 0.15, ko.IMEX, 2, prec=32,
                        status=True, switch_tol=float(sw))
    assert st[0] == (5, 0) and res[0][1] == float(np.float64(T0))   # switched at once, T kept
    assert st[1] == (0, 2)


def test_items_xi_pairs_descent_matches_oracle():
    """In the centre-symmetric subspace the column items work on column pairs (2p+1, 2p+2): a
    ragged batch of odd-in-x loops (Kx = 10, even, and Kx = 5, odd: the last pair has no second
    column) against the oracle's descent in the subspace, five IMEX steps, FP64."""
    for nx, nss in ((32, [32, 8, 64]), (16, [16, 128])):
        loops = []
        for i, n in enumerate(nss):
            u, T, _ = spectral_loop(20 + i, nx, 39.0, ns=n, T_range=(30.0, 50.0), symmetric=True)
            loops.append((u, T))
        res = run_batch(harness_exe(), loops, 39.0, 0.15, ko.IMEX, 5, xi=1)
        for (u, T), (a, c, g) in zip(loops, res):
            ref = ko.descend(u, T, 39.0, 0.15, ko.IMEX, 5, xi=True)
            assert rel(g, ref["u"]) <= 1e-12 and abs(c - ref["T"]) <= 1e-12 * ref["T"]
            assert abs(a - np.sqrt(ko.residual(u, T, 39.0, xi=True)["J"])) <= 1e-12 * a
