"""ctypes binding of the C ABI in ``include/ks_loop.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but turn
torch tensors / NumPy arrays into pointers, check the return code and raise ``KsError`` with
``ks_last_error()``.  All arithmetic runs in ``libks_loop.so`` on the GPU; if the library is
missing the import fails loudly (there is no CPU path).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libks_loop.so")

KS_FP64, KS_FP32, KS_MIXED = 0, 1, 2
KS_EXPLICIT, KS_IMEX = 0, 1
KS_OK, KS_ERR_ARG, KS_ERR_CUDA, KS_ERR_OOM, KS_ERR_TIMEOUT, KS_ERR_STATE = 0, -1, -2, -3, -4, -5
KS_RUNNING, KS_CONVERGED, KS_STEP_CAP, KS_STALLED, KS_DIVERGED = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "running", 1: "converged", 2: "step_cap", 3: "stalled", 4: "diverged"}

_EXPORTS = ("ks_loop_create", "ks_destroy", "ks_residual", "ks_adjoint_grad", "ks_descend",
            "ks_set_state", "ks_step", "ks_get_state", "ks_last_error", "ks_version",
            "ks_config_sizeof", "ks_profile", "ks_profile_read", "ks_set_option", "ks_get_option",
            "ks_residual_noalloc", "ks_get_history", "ks_autotune", "ks_band_size",
            "ks_get_band", "ks_set_band", "ks_probe_peak", "ks_dns", "ks_dns_segments")


class KsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ks_loop error {code}: {msg}")
        self.code = code


class ks_config(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("nx", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("ns", ctypes.POINTER(ctypes.c_int)),
        ("mode", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("dtau", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("switch_tol", ctypes.c_double),
        ("max_steps", ctypes.c_longlong),
        ("chunk", ctypes.c_int),
        ("autotune", ctypes.c_int),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libks_loop.so (built in-tree by ``paper_2007_06427_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2007_06427_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    lib.ks_loop_create.argtypes = [ctypes.POINTER(ks_config), ctypes.POINTER(vp)]
    lib.ks_destroy.argtypes = [vp]
    lib.ks_residual.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ks_adjoint_grad.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ks_descend.argtypes = [vp, vp, vp, i64, dp, vp, vp, vp, vp]
    lib.ks_set_state.argtypes = [vp, vp, vp, vp]
    lib.ks_step.argtypes = [vp, i64, dp, vp]
    lib.ks_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.ks_profile.argtypes = [vp, i32]
    lib.ks_set_option.argtypes = [vp, ctypes.c_char_p, i64]
    lib.ks_get_option.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong)]
    lib.ks_residual_noalloc.argtypes = [dp, i32, i32, vp, dp, vp, vp, vp]
    lib.ks_get_history.argtypes = [vp, i32, vp, vp, vp, i32]
    lib.ks_autotune.argtypes = [vp]
    lib.ks_band_size.argtypes = [vp]
    lib.ks_band_size.restype = i64
    lib.ks_get_band.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ks_set_band.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ks_profile_read.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    lib.ks_probe_peak.argtypes = [i32, i32, vp, vp]
    lib.ks_dns.argtypes = [dp, i32, i32, dp, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.ks_dns_segments.argtypes = [i32, i64, dp, vp, i32, vp, vp, vp, vp, vp]
    for f in ("ks_loop_create", "ks_destroy", "ks_residual", "ks_adjoint_grad", "ks_descend",
              "ks_set_state", "ks_step", "ks_get_state", "ks_profile", "ks_profile_read",
              "ks_set_option", "ks_get_option", "ks_residual_noalloc", "ks_get_history",
              "ks_autotune", "ks_get_band", "ks_set_band", "ks_probe_peak", "ks_dns",
              "ks_dns_segments"):
        getattr(lib, f).restype = i32
    lib.ks_last_error.restype = ctypes.c_char_p
    lib.ks_version.restype = ctypes.c_char_p
    lib.ks_config_sizeof.restype = ctypes.c_ulonglong
    if lib.ks_config_sizeof() != ctypes.sizeof(ks_config):
        raise ImportError("ks_config layout mismatch between the binding and the library")
    _lib = lib
    return lib


def _check(rc: int):
    if rc != KS_OK:
        raise KsError(rc, ks_last_error())


def _ptr(x) -> Optional[int]:
    """Data pointer of a torch tensor or NumPy array (None passes through as NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- the C entry points, same names -------------------------------------------------------

def ks_last_error() -> str:
    return load_library().ks_last_error().decode()


def ks_version() -> str:
    return load_library().ks_version().decode()


def ks_config_sizeof() -> int:
    return int(load_library().ks_config_sizeof())


def ks_loop_create(L: float, nx: int, ns: Sequence[int], mode: int = KS_FP64,
                   scheme: int = KS_IMEX, dtau: float = 0.15, tol: float = 1e-10,
                   switch_tol: float = 0.0, max_steps: int = 1_000_000, chunk: int = 1000,
                   autotune: int = 0) -> int:
    lib = load_library()
    nsa = (ctypes.c_int * len(ns))(*[int(v) for v in ns])
    cfg = ks_config(float(L), int(nx), len(ns), nsa, int(mode), int(scheme), float(dtau),
                    float(tol), float(switch_tol), int(max_steps), int(chunk), int(autotune))
    h = ctypes.c_void_p()
    _check(lib.ks_loop_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def ks_destroy(h) -> None:
    _check(load_library().ks_destroy(h))


def ks_residual(h, u, T, r=None, J=None, stream=None) -> None:
    _check(load_library().ks_residual(h, _ptr(u), _ptr(T), _ptr(r), _ptr(J), _stream(stream)))


def ks_adjoint_grad(h, u, T, G, dJdT=None, stream=None) -> None:
    _check(load_library().ks_adjoint_grad(h, _ptr(u), _ptr(T), _ptr(G), _ptr(dJdT),
                                          _stream(stream)))


def ks_descend(h, u, T, max_steps: int = -1, tol: float = -1.0, steps=None, sqrtJ=None,
               status=None, stream=None) -> None:
    _check(load_library().ks_descend(h, _ptr(u), _ptr(T), int(max_steps), float(tol),
                                     _ptr(steps), _ptr(sqrtJ), _ptr(status), _stream(stream)))


def ks_set_state(h, u, T, stream=None) -> None:
    _check(load_library().ks_set_state(h, _ptr(u), _ptr(T), _stream(stream)))


def ks_step(h, nsteps: int, tol: float = -1.0, stream=None) -> None:
    _check(load_library().ks_step(h, int(nsteps), float(tol), _stream(stream)))


def ks_get_state(h, u=None, T=None, steps=None, sqrtJ=None, status=None, stream=None) -> None:
    _check(load_library().ks_get_state(h, _ptr(u), _ptr(T), _ptr(steps), _ptr(sqrtJ),
                                       _ptr(status), _stream(stream)))


def ks_set_option(h, key: str, value: int) -> None:
    _check(load_library().ks_set_option(h, key.encode(), int(value)))


def ks_get_option(h, key: str) -> int:
    v = ctypes.c_longlong()
    _check(load_library().ks_get_option(h, key.encode(), ctypes.byref(v)))
    return v.value


def ks_residual_noalloc(L: float, nx: int, ns: int, u, T: float, r=None, J=None,
                        stream=None) -> None:
    """Residual of one double loop with no device allocation (device buffers only)."""
    _check(load_library().ks_residual_noalloc(float(L), int(nx), int(ns), _ptr(u), float(T),
                                              _ptr(r), _ptr(J), _stream(stream)))


def ks_band_size(h) -> int:
    return int(load_library().ks_band_size(h))


def ks_get_band(h, band, T=None, prec=None, steps=None, stream=None) -> None:
    _check(load_library().ks_get_band(h, _ptr(band), _ptr(T), _ptr(prec), _ptr(steps),
                                      _stream(stream)))


def ks_set_band(h, band, T, prec=None, steps=None, stream=None) -> None:
    _check(load_library().ks_set_band(h, _ptr(band), _ptr(T), _ptr(prec), _ptr(steps),
                                      _stream(stream)))


def ks_autotune(h) -> None:
    _check(load_library().ks_autotune(h))


def ks_get_history(h, b: int):
    """(steps, sqrtJ, prec) arrays recorded by the last ks_descend for loop b."""
    lib = load_library()
    n = lib.ks_get_history(h, int(b), None, None, None, 0)
    if n < 0:
        raise KsError(n, ks_last_error())
    st = np.zeros(n, dtype=np.int64)
    sq = np.zeros(n, dtype=np.float64)
    pr = np.zeros(n, dtype=np.int32)
    if n:
        lib.ks_get_history(h, int(b), st.ctypes.data, sq.ctypes.data, pr.ctypes.data, n)
    return st, sq, pr


def ks_probe_peak(precision: int, iters: int = 0, stream=None) -> float:
    """Measured FMA peak of the current device in TFLOP/s (KS_FP64 or KS_FP32)."""
    if iters <= 0:
        iters = 500 if precision == KS_FP64 else 10000   # ~2 ms and ~0.7 ms per launch on GB300
    v = ctypes.c_double()
    _check(load_library().ks_probe_peak(int(precision), int(iters), ctypes.byref(v), _stream(stream)))
    return v.value


def ks_dns(L: float, nx: int, batch: int, dt: float, nsteps: int, save_every: int, symmetric: bool,
           u0, u_saved=None, norms=None, u_end=None, stream=None) -> None:
    _check(load_library().ks_dns(L, nx, batch, dt, nsteps, save_every, int(bool(symmetric)),
                                 _ptr(u0), _ptr(u_saved), _ptr(norms), _ptr(u_end), _stream(stream)))


def ks_dns_segments(nx: int, nsave: int, dts: float, us, a_idx, T, ns, out, stream=None) -> None:
    """a_idx, T and ns are host arrays (int32, float64, int32), one entry per loop."""
    a_idx = np.ascontiguousarray(a_idx, dtype=np.int32)
    T = np.ascontiguousarray(T, dtype=np.float64)
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    _check(load_library().ks_dns_segments(nx, nsave, dts, _ptr(us), len(a_idx), _ptr(a_idx), _ptr(T),
                                          _ptr(ns), _ptr(out), _stream(stream)))


def ks_profile(h, enable: bool) -> None:
    _check(load_library().ks_profile(h, int(bool(enable))))


def ks_profile_read(h, reset: bool = False):
    """Returns ({kind: (ms, launches)}, total_launches)."""
    lib = load_library()
    n = 64
    names = ctypes.create_string_buffer(n * 48)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    tot = ctypes.c_longlong()
    k = lib.ks_profile_read(h, n, names, ms, cnt, ctypes.byref(tot), int(bool(reset)))
    if k < 0:
        raise KsError(k, ks_last_error())
    raw = names.raw
    out = {}
    for i in range(min(k, n)):
        nm = raw[i * 48:(i + 1) * 48].split(b"\0", 1)[0].decode()
        out[nm] = (ms[i], cnt[i])
    return out, tot.value


# ---- convenience owner of a handle ---------------------------------------------------------

class KSLoop:
    """Owns one handle; buffers are torch tensors or NumPy arrays supplied by the caller."""

    def __init__(self, L: float, nx: int, ns: Sequence[int], mode: int = KS_FP64,
                 scheme: int = KS_IMEX, dtau: float = 0.15, tol: float = 1e-10,
                 switch_tol: float = 0.0, max_steps: int = 1_000_000, chunk: int = 1000,
                 autotune: int = 0):
        self.L, self.nx, self.ns = float(L), int(nx), [int(v) for v in ns]
        self.mode, self.scheme, self.dtau = int(mode), int(scheme), float(dtau)
        self.handle = ks_loop_create(L, nx, ns, mode, scheme, dtau, tol, switch_tol, max_steps,
                                     chunk, autotune)

    @property
    def batch(self) -> int:
        return len(self.ns)

    @property
    def gridpoints(self) -> int:
        return int(sum(self.ns)) * self.nx

    @property
    def np_dtype(self):
        return np.float32 if self.mode == KS_FP32 else np.float64

    def close(self):
        if getattr(self, "handle", None):
            ks_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
