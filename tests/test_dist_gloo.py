"""Multi-process (world size 2, gloo, CPU) checks of the sharding and the
collectives the multi-GPU benchmark and gradient paths use."""
import os
import socket

import numpy as np
import pytest

from paper_2105_01796_gb300 import dist as kdist
from paper_2105_01796_gb300 import synth


def test_shards_partition_and_balance_states():
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 5000))
    o = ev["offsets"]
    for world in (1, 2, 3, 8):
        ranges = [kdist.shard_range(5000, r, world, o) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == 5000
        for a, b in zip(ranges, ranges[1:]):
            assert a[1] == b[0]
        states = [int(o[e] - o[b]) for b, e in ranges]
        assert max(states) - min(states) <= 31 + 1   # at most about one track apart
        eq = [kdist.shard_range(5000, r, world) for r in range(world)]
        sizes = [e - b for b, e in eq]
        assert sum(sizes) == 5000 and max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ev = synth.make_event(synth.scaled(synth.WORKLOADS["uneven30_1m"], 1000))
        b, e = kdist.shard_range(1000, rank, world, ev["offsets"])
        # per-rank "time" and a per-surface gradient of this shard
        t = kdist.max_over_ranks(10.0 + rank)
        g = torch.full((120,), float(e - b), dtype=torch.float64)
        kdist.sum_over_ranks(g)
        results[rank] = (b, e, t, float(g[0]), float(g[-1]))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_collectives():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (b0, e0, t0, g0, h0), (b1, e1, t1, g1, h1) = results[0], results[1]
    assert b0 == 0 and e0 == b1 and e1 == 1000
    assert t0 == t1 == 11.0                     # max over ranks
    assert g0 == g1 == h0 == h1 == 1000.0       # sum of the shards' track counts


def _grad_worker(rank, world, port, results):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 60))
        b, e = kdist.shard_range(60, rank, world, ev["offsets"])
        shard = synth.subset(ev, np.arange(b, e))
        _, ga = oracle.chi2_gradient_fd(shard, n_threads=1)
        g = torch.from_numpy(np.ascontiguousarray(ga.ravel()))
        kdist.sum_over_ranks(g)
        results[rank] = g.numpy().copy()
    finally:
        dist.destroy_process_group()


def test_sharded_alignment_gradient_sums_to_the_full_gradient():
    """The alignment gradient of the summed chi2 over a batch equals the sum of
    the shards' gradients: each rank takes the oracle's gradient of its track
    range and one all-reduce (120 + 6 values here) adds them."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    ev = synth.make_event(synth.scaled(synth.WORKLOADS["align20_100k"], 60))
    _, full = oracle.chi2_gradient_fd(ev, n_threads=1)
    for r in range(2):
        got = results[r].reshape(full.shape)
        assert np.max(np.abs(got - full)) <= 1e-6 * np.max(np.abs(full))
