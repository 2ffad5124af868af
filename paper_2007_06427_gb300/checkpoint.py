"""Checkpoint and resume of a descent (host side).

A checkpoint is an .npz file holding the handle's configuration (L, Nx, the Ns list, mode,
scheme, dtau, tolerances), its descent knobs (``KNOBS``: symmetry, extrapolation, stall window
and threshold, mixed finish, chunk, each precision's launch form, graph replay), the band state
of every loop (ks_get_band: the Fourier coefficients u_hat of Eq. 2D_Fourier, widened to
double), T, the step counters, the precision each loop descends in, each loop's status and its
convergence history.

Resuming creates a handle with the same configuration and knobs and installs the band with
ks_set_band.  What is and is not restored:
* every loop that was running continues bit for bit as in an uninterrupted descent (same
  band, T, counters, precision and knobs);
* ks_set_band restarts every loop as running, so the saved statuses and histories are returned
  to the caller (``resume(..., info=True)``) rather than reinstalled: a converged loop freezes
  again before its next step (its sqrt(J) is below tol), a stalled or diverged one steps on
  unless the caller leaves it out;
* with the "extrapolate" knob the anchors of the extrapolation are not saved: a resumed descent
  takes new anchors at its first read-back, so its later extrapolations can differ from an
  uninterrupted run's.
"""
from __future__ import annotations

import numpy as np

from . import ks_loop as K

_KEYS = ("L", "nx", "ns", "mode", "scheme", "dtau", "tol", "switch_tol", "band", "T", "prec",
         "steps", "status", "version")
VERSION = 2
# knobs of ks_set_option that change how the descent proceeds (saved and restored)
KNOBS = ("symmetry", "extrapolate", "extrapolate_start_ppm", "extrapolate_drop_ppm",
         "stall_window", "stall_drop_ppm", "finish_f32_adjoint", "switch_probe",
         "switch_probe_steps", "chunk", "path_f64", "path_f32", "graph")


def save(loop: "K.KSLoop", path: str, tol: float = 1e-10, switch_tol: float = 0.0) -> None:
    n = K.ks_band_size(loop.handle)
    band = np.zeros(2 * n, dtype=np.float64)
    T = np.zeros(loop.batch, dtype=np.float64)
    prec = np.zeros(loop.batch, dtype=np.int32)
    steps = np.zeros(loop.batch, dtype=np.int64)
    K.ks_get_band(loop.handle, band, T, prec, steps)
    status = np.zeros(loop.batch, dtype=np.int32)
    K.ks_get_state(loop.handle, None, None, None, None, status)
    knobs = {f"knob_{k}": K.ks_get_option(loop.handle, k) for k in KNOBS}
    hist = {}
    for b in range(loop.batch):
        hs, hq, hp = K.ks_get_history(loop.handle, b)
        hist[f"hist_steps_{b}"] = hs
        hist[f"hist_sqrtJ_{b}"] = hq
        hist[f"hist_prec_{b}"] = hp
    np.savez(path, L=loop.L, nx=loop.nx, ns=np.asarray(loop.ns, dtype=np.int64), mode=loop.mode,
             scheme=loop.scheme, dtau=loop.dtau, tol=tol, switch_tol=switch_tol, band=band, T=T,
             prec=prec, steps=steps, status=status, version=VERSION, **knobs, **hist)


def resume(path: str, info: bool = False, **create_kw):
    """A new handle holding the checkpointed descent, its knobs restored (raises ValueError on a
    bad file).  With info, returns (handle, {"status": [...], "history": {b: (steps, sqrtJ,
    prec)}}) as saved."""
    with np.load(path) as z:
        missing = [k for k in _KEYS if k not in z.files]
        if missing:
            raise ValueError(f"checkpoint {path} lacks {missing}")
        if int(z["version"]) != VERSION:
            raise ValueError(f"checkpoint version {int(z['version'])} != {VERSION}")
        ns = [int(v) for v in z["ns"]]
        loop = K.KSLoop(float(z["L"]), int(z["nx"]), ns, int(z["mode"]), int(z["scheme"]),
                        float(z["dtau"]), tol=float(z["tol"]), switch_tol=float(z["switch_tol"]),
                        **create_kw)
        band = np.ascontiguousarray(z["band"], dtype=np.float64)
        if band.size != 2 * K.ks_band_size(loop.handle) or z["T"].size != loop.batch:
            loop.close()
            raise ValueError(f"checkpoint {path} does not match its own configuration")
        for k in KNOBS:
            if f"knob_{k}" in z.files:
                K.ks_set_option(loop.handle, k, int(z[f"knob_{k}"]))
        K.ks_set_band(loop.handle, band, np.ascontiguousarray(z["T"], dtype=np.float64),
                      np.ascontiguousarray(z["prec"], dtype=np.int32),
                      np.ascontiguousarray(z["steps"], dtype=np.int64))
        saved = {"status": [int(v) for v in z["status"]],
                 "history": {b: (z[f"hist_steps_{b}"], z[f"hist_sqrtJ_{b}"], z[f"hist_prec_{b}"])
                             for b in range(loop.batch) if f"hist_steps_{b}" in z.files}}
    return (loop, saved) if info else loop
