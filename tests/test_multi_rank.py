"""Multi-rank path on CPU: two gloo ranks split a ragged batch with shard.partition, each
descends its loops (the CPU oracle stands in for the per-rank GPU descent), and the gathered
result equals a serial descent of the whole batch, loop for loop."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2007_06427_gb300 import shard
from paper_2007_06427_gb300.inputs import make_loops


def _batch():
    return make_loops("ragged_small", 16, 22.0, range(5), ns_choices=(8, 16, 32),
                      T_range=(20.0, 60.0), scheme=1, dtau=0.15)


def _descend(u, T, ns, nx, L):
    from oracle import ks_oracle as ko
    res, off = [], 0
    for n, t in zip(ns, T):
        out = ko.descend(u[off:off + n * nx].reshape(n, nx), float(t), L, 0.15, ko.IMEX, 6)
        res.append(out)
        off += n * nx
    return res


def _worker(rank, world, port, outq):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _batch()
    parts = shard.partition(w.ns, w.nx, world)
    mine = parts[rank]
    u, T, ns = shard.local_batch(w.packed(), w.ns, w.nx, w.T0, mine)
    outs = _descend(u, T, ns, w.nx, w.L)
    local = {b: {"u": o["u"].ravel(), "T": o["T"], "steps": o["steps"]} for b, o in zip(mine, outs)}
    allres = shard.gather(local)
    if rank == 0:
        uu, TT = shard.scatter_back(allres, w.ns, w.nx)
        outq.put((uu, TT, [len(p) for p in parts]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_covers_and_balances():
    ns = [256, 32, 128, 64, 256, 32, 32, 128, 64]
    parts = shard.partition(ns, 64, 3)
    flat = sorted(b for p in parts for b in p)
    assert flat == list(range(len(ns)))
    loads = [sum(ns[b] for b in p) for p in parts]
    assert max(loads) - min(loads) <= max(ns)
    assert shard.partition(ns, 64, 1) == [list(range(len(ns)))]


def test_two_gloo_ranks_match_serial_descent():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    uu, TT, sizes = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = _batch()
    ref = _descend(w.packed(), w.T0, w.ns, w.nx, w.L)
    ref_u = np.concatenate([o["u"].ravel() for o in ref])
    ref_T = np.array([o["T"] for o in ref])
    np.testing.assert_array_equal(uu, ref_u)
    np.testing.assert_array_equal(TT, ref_T)
    assert sum(sizes) == w.batch and min(sizes) >= 1


def test_more_ranks_than_loops_and_round_trip():
    """Ranks without loops get an empty list; each rank's slice of the packed field and the
    reassembly in batch order invert each other; a missing loop is reported."""
    ns, nx = [64, 32, 128], 16
    parts = shard.partition(ns, nx, 5)
    assert len(parts) == 5 and sorted(b for p in parts for b in p) == [0, 1, 2]
    assert sum(1 for p in parts if not p) == 2
    rng = np.random.default_rng(0)
    u = rng.standard_normal(sum(ns) * nx)
    T = [30.0, 40.0, 50.0]
    results = {}
    for p in parts:
        ul, Tl, nsl = shard.local_batch(u, ns, nx, T, p)
        assert ul.size == sum(n * nx for n in nsl) and list(Tl) == [T[b] for b in p]
        o = 0
        for b, n in zip(p, nsl):
            results[b] = {"u": ul[o:o + n * nx], "T": Tl[p.index(b)]}
            o += n * nx
    u2, T2 = shard.scatter_back(results, ns, nx)
    assert np.array_equal(u2, u) and list(T2) == T
    del results[1]
    with pytest.raises(ValueError, match="1"):
        shard.scatter_back(results, ns, nx)
    with pytest.raises(ValueError):
        shard.partition(ns, nx, 0)
