"""Checkpoint and resume of a descent (host side).

A checkpoint is an .npz file holding the handle's configuration (L, Nx, the Ns list, mode,
scheme, dtau, tolerances), the band state of every loop (ks_get_band: the Fourier
coefficients u_hat of Eq. 2D_Fourier, widened to double), T, the step counters, the
precision each loop descends in, and each loop's convergence history.  Resuming creates a
handle with the same configuration and installs the band with ks_set_band, so the continued
descent is bit-identical to an uninterrupted one.  (With the "extrapolate" knob the anchors of
the extrapolation are not saved: a resumed descent takes new anchors at its first read-back, so
its later extrapolations can differ from an uninterrupted run's.)
"""
from __future__ import annotations

import numpy as np

from . import ks_loop as K

_KEYS = ("L", "nx", "ns", "mode", "scheme", "dtau", "tol", "switch_tol", "band", "T", "prec",
         "steps", "version")
VERSION = 1


def save(loop: "K.KSLoop", path: str, tol: float = 1e-10, switch_tol: float = 0.0) -> None:
    n = K.ks_band_size(loop.handle)
    band = np.zeros(2 * n, dtype=np.float64)
    T = np.zeros(loop.batch, dtype=np.float64)
    prec = np.zeros(loop.batch, dtype=np.int32)
    steps = np.zeros(loop.batch, dtype=np.int64)
    K.ks_get_band(loop.handle, band, T, prec, steps)
    hist = {}
    for b in range(loop.batch):
        hs, hq, hp = K.ks_get_history(loop.handle, b)
        hist[f"hist_steps_{b}"] = hs
        hist[f"hist_sqrtJ_{b}"] = hq
        hist[f"hist_prec_{b}"] = hp
    np.savez(path, L=loop.L, nx=loop.nx, ns=np.asarray(loop.ns, dtype=np.int64), mode=loop.mode,
             scheme=loop.scheme, dtau=loop.dtau, tol=tol, switch_tol=switch_tol, band=band, T=T,
             prec=prec, steps=steps, version=VERSION, **hist)


def resume(path: str, **create_kw) -> "K.KSLoop":
    """A new handle holding the checkpointed descent (raises ValueError on a bad file)."""
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
        K.ks_set_band(loop.handle, band, np.ascontiguousarray(z["T"], dtype=np.float64),
                      np.ascontiguousarray(z["prec"], dtype=np.int32),
                      np.ascontiguousarray(z["steps"], dtype=np.int64))
    return loop
