"""The autotuner picks a launch shape by timing; every candidate computes the same thing, so a
tuned handle reproduces an untuned one bit for bit.  The on-disk cache is written once and
reused."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_06427_gb300 import ks_loop as K
from paper_2007_06427_gb300.inputs import spectral_loop

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [K.KS_FP64, K.KS_FP32, K.KS_MIXED])
def test_tuned_handle_reproduces_default(mode, tmp_path, monkeypatch):
    monkeypatch.setenv("KS_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    L, nx, nss = 22.0, 64, [64, 128, 32]
    us, Ts = [], []
    for i, n in enumerate(nss):
        u, T, _ = spectral_loop(i, nx, L, ns=n, T_range=(20.0, 80.0))
        us.append(u)
        Ts.append(T)
    dt = torch.float32 if mode == K.KS_FP32 else torch.float64
    outs = []
    for tune in (0, 1):
        u = torch.tensor(np.concatenate([a.ravel() for a in us]), device="cuda").to(dt)
        T = torch.tensor(Ts, dtype=torch.float64, device="cuda")
        with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, autotune=tune, chunk=6) as h:
            if tune:
                assert K.ks_get_option(h.handle, "path") in (0, 1, 2)
                assert K.ks_get_option(h.handle, "cluster_threads") in (128, 256)
            K.ks_descend(h.handle, u, T, 15, 0.0)
        outs.append((u.cpu(), T.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    lines = open(tmp_path / "tune.txt").read().strip().splitlines()
    assert len(lines) == 1 and "|" in lines[0]
    # a second tuned handle of the same shape reads the cache instead of timing again
    with K.KSLoop(L, nx, nss, mode, K.KS_IMEX, 0.15, autotune=1) as h:
        pass
    assert len(open(tmp_path / "tune.txt").read().strip().splitlines()) == 1


def test_invalid_cache_entry_is_ignored(tmp_path, monkeypatch):
    """A cache line naming a launch shape the tuner never tries (here 32 threads, which the
    cluster kernel cannot run) is ignored: the handle times the candidates again and appends a
    valid entry."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("KS_AUTOTUNE_CACHE", str(cache))
    L, nx, nss = 22.0, 32, [32]
    with K.KSLoop(L, nx, nss, K.KS_FP64, K.KS_IMEX, 0.15, autotune=1):
        pass
    key, choice = cache.read_text().strip().split("|")
    path, cluster, threads = map(int, choice.split())
    cache.write_text(f"{key}|0 {cluster} 32\n")
    with K.KSLoop(L, nx, nss, K.KS_FP64, K.KS_IMEX, 0.15, autotune=1) as h:
        assert K.ks_get_option(h.handle, "cluster_threads") in (128, 256)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 2 and lines[0].endswith(" 32")
    assert int(lines[1].split("|")[1].split()[2]) in (128, 256)


def test_default_launch_path_rule():
    """The launch form chosen at create without tuning, per precision (P = Nx * max Ns): four
    launches per step for ragged batches of 64 or more loops; in double once P >= 16384, or
    P >= 8192 in batches of 8 or more, or with 1 or 2 CTAs per loop's cluster on P >= 4096; in
    float once P >= 32768, or P >= 16384 in batches of 64 or more; the cluster-resident kernel
    otherwise.  "path" reads the bulk precision's form (float for mixed handles)."""
    from paper_2007_06427_gb300.inputs import workload
    rg = workload("ragged256_64xNs", batch=64)
    for mode in (K.KS_FP64, K.KS_FP32, K.KS_MIXED):
        with K.KSLoop(rg.L, rg.nx, rg.ns, mode) as h:
            assert K.ks_get_option(h.handle, "path") == 2, mode
    with K.KSLoop(22.0, 64, [64] * 256, K.KS_FP64) as h:
        assert K.ks_get_option(h.handle, "cluster_f64") in (1, 2)
        assert K.ks_get_option(h.handle, "path") == 2
    for mode in (K.KS_FP32, K.KS_MIXED):
        with K.KSLoop(22.0, 64, [64] * 256, mode) as h:
            assert K.ks_get_option(h.handle, "path") == 0, mode
    with K.KSLoop(22.0, 32, [32] * 256, K.KS_FP64) as h:     # 1024-point loops
        assert K.ks_get_option(h.handle, "path") == 0
    with K.KSLoop(22.0, 64, [128], K.KS_FP64) as h:          # the single loop
        assert K.ks_get_option(h.handle, "path") == 0
        assert K.ks_get_option(h.handle, "cluster_f64") == 16
    with K.KSLoop(22.0, 64, [128] * 8, K.KS_FP64) as h:      # 8192 points, 8 loops
        assert K.ks_get_option(h.handle, "path") == 2
    with K.KSLoop(22.0, 64, [256], K.KS_MIXED) as h:         # 16384 points, one loop
        assert K.ks_get_option(h.handle, "path") == 0
        assert K.ks_get_option(h.handle, "path_f32") == 0
        assert K.ks_get_option(h.handle, "path_f64") == 2
    with K.KSLoop(44.0, 128, [128] * 64, K.KS_FP32) as h:    # 16384 points, 64 loops
        assert K.ks_get_option(h.handle, "path") == 2
    for mode in (K.KS_FP64, K.KS_FP32, K.KS_MIXED):          # the large domain, 8 loops
        with K.KSLoop(100.0, 256, [1024] * 8, mode) as h:
            assert K.ks_get_option(h.handle, "path_f64") == 2, mode
            assert K.ks_get_option(h.handle, "path_f32") == 2, mode
    with K.KSLoop(22.0, 64, [256], K.KS_MIXED) as h:
        K.ks_set_option(h.handle, "path", 1)
        assert (K.ks_get_option(h.handle, "path_f64"), K.ks_get_option(h.handle, "path_f32")) == (1, 1)
        K.ks_set_option(h.handle, "path_f64", 0)
        assert (K.ks_get_option(h.handle, "path_f64"), K.ks_get_option(h.handle, "path_f32")) == (0, 1)


def test_cluster_block_width_rule():
    """Threads per CTA of the cluster kernel: the 128 work threads plus one warp for the step
    scalars for a float state always, for a double state when no transform of its plan has more
    than 128 butterflies a pass (the single 64 x 128 loop on 16 CTAs: 8 rows and 2 columns of 128
    per CTA); the 256-thread width has no extra warp.  Every width gives the same bits (the
    launch-form and autotune tests compare them)."""
    with K.KSLoop(22.0, 64, [128], K.KS_MIXED) as h:
        assert K.ks_get_option(h.handle, "cluster_threads") == 128
        assert K.ks_get_option(h.handle, "cluster_block_f64") == 160
        assert K.ks_get_option(h.handle, "cluster_block_f32") == 160
    with K.KSLoop(100.0, 256, [1024], K.KS_FP64) as h:       # 256-point rows, 1024-point columns
        if K.ks_get_option(h.handle, "cluster_f64"):
            assert K.ks_get_option(h.handle, "cluster_block_f64") == 128
