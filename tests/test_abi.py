"""C ABI checks that need no GPU: the library builds, loads, exports every function declared
in include/ks_loop.h, agrees on the ks_config layout, and rejects bad arguments (or the
missing device) with an error code instead of computing anything on the CPU."""
import os
import re

import pytest

from paper_2007_06427_gb300 import ks_loop as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ks_loop.h")).read()
    return sorted(set(re.findall(r"^KS_API\s+[\w\s\*]+?\b(ks_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(K.LIB_PATH):
        from paper_2007_06427_gb300 import build
        build.build()
    return K.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ks_loop_create", "ks_residual", "ks_adjoint_grad", "ks_descend", "ks_destroy"):
        assert f in names


def test_every_option_key_is_documented():
    """Every key ks_set_option / ks_get_option accept is described in the header."""
    src = open(os.path.join(ROOT, "paper_2007_06427_gb300", "csrc", "ks_loop.cu")).read()
    hdr = open(os.path.join(ROOT, "include", "ks_loop.h")).read()
    keys = sorted(set(re.findall(r'k == "([a-z0-9_]+)"', src)))
    assert len(keys) > 20
    assert [k for k in keys if f'"{k}"' not in hdr] == []


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(K._EXPORTS)


def test_config_layout(lib):
    import ctypes
    assert lib.ks_config_sizeof() == ctypes.sizeof(K.ks_config)


@pytest.mark.parametrize("kw", [
    dict(L=22.0, nx=48, ns=[32]),          # nx not a power of two
    dict(L=22.0, nx=4, ns=[32]),           # nx too small
    dict(L=22.0, nx=2048, ns=[32]),        # nx too large
    dict(L=22.0, nx=32, ns=[24]),          # ns not a power of two
    dict(L=22.0, nx=32, ns=[32, 2048]),    # one ns too large
    dict(L=-1.0, nx=32, ns=[32]),          # L <= 0
    dict(L=22.0, nx=32, ns=[32], dtau=0.0),
    dict(L=22.0, nx=32, ns=[32], mode=7),
    dict(L=22.0, nx=32, ns=[32], scheme=3),
])
def test_bad_arguments_rejected(lib, kw):
    with pytest.raises(K.KsError) as e:
        K.ks_loop_create(**kw)
    assert e.value.code == K.KS_ERR_ARG


def test_null_handle_rejected(lib):
    import numpy as np
    with pytest.raises(K.KsError) as e:
        K.ks_residual(None, np.zeros(4), np.zeros(1))
    assert e.value.code == K.KS_ERR_ARG


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(K.KsError) as e:
        K.ks_loop_create(22.0, 32, [32])
    assert e.value.code == K.KS_ERR_CUDA


def test_probe_rejects_bad_arguments_and_needs_a_device(lib):
    import ctypes
    v = ctypes.c_double(0.0)
    assert lib.ks_probe_peak(7, 10, ctypes.byref(v), None) == K.KS_ERR_ARG
    assert lib.ks_probe_peak(K.KS_FP64, 0, ctypes.byref(v), None) == K.KS_ERR_ARG
    assert lib.ks_probe_peak(K.KS_FP64, 10, None, None) == K.KS_ERR_ARG
    import torch
    if not torch.cuda.is_available():
        assert lib.ks_probe_peak(K.KS_FP64, 10, ctypes.byref(v), None) == K.KS_ERR_CUDA
        assert v.value == 0.0


@pytest.mark.parametrize("kw", [
    dict(L=0.0), dict(dt=-0.25), dict(nx=48), dict(nx=2048), dict(batch=0), dict(nsteps=-1),
    dict(save_every=0), dict(u0=None),
])
def test_dns_rejects_bad_arguments(lib, kw):
    import numpy as np
    a = dict(L=22.0, nx=32, batch=1, dt=0.25, nsteps=4, save_every=1, symmetric=False,
             u0=np.zeros(32))
    a.update(kw)
    with pytest.raises(K.KsError) as e:
        K.ks_dns(**a)
    assert e.value.code == K.KS_ERR_ARG


def test_dns_segments_rejects_bad_arguments(lib):
    import numpy as np
    us = np.zeros((10, 8))
    out = np.zeros(8 * 8)
    good = dict(nx=8, nsave=10, dts=0.5, us=us, a_idx=[0], T=[3.0], ns=[8], out=out)
    for kw in (dict(nsave=1), dict(dts=0.0), dict(T=[-1.0]), dict(ns=[0]), dict(a_idx=[-1]),
               dict(T=[5.5]), dict(us=None)):
        a = dict(good)
        a.update(kw)
        with pytest.raises(K.KsError) as e:
            K.ks_dns_segments(**a)
        assert e.value.code == K.KS_ERR_ARG, kw


def test_dns_needs_a_device(lib):
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(K.KsError) as e:
        K.ks_dns(22.0, 32, 1, 0.25, 4, 1, False, np.zeros(32))
    assert e.value.code == K.KS_ERR_CUDA
    with pytest.raises(K.KsError) as e:       # the last instant 5 * 7/8 needs samples 8 and 9
        K.ks_dns_segments(8, 10, 0.5, np.zeros((10, 8)), [0], [5.0], [8], np.zeros(64))
    assert e.value.code == K.KS_ERR_CUDA
