"""Multi-rank host logic on CPU (world size 2, gloo): scenes sharded across ranks with no
data-path collective give exactly the single-process results -- final states, and the
losses and gradients of a forward+backward run gathered through the rendezvous store --
the benchmark's max-over-ranks timing reduction works, and a rank that fails before
reporting its shard is detected by the others through the rendezvous store within a
deadline (no collective hangs).  The per-rank work is the FP64 oracle (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1910_00935_gb300 import scenes
from paper_1910_00935_gb300.sharding import RankFailure, collect_shards, shard_scenes, subset


def test_shards_partition_and_balance():
    counts = [5000, 100, 2000, 2000, 7000, 300, 300, 4000]
    for world in (1, 2, 3, 4):
        shards = [shard_scenes(counts, world, r) for r in range(world)]
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(counts)))          # a partition
        loads = [sum(counts[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(counts)     # greedy balance bound
        assert shards == [shard_scenes(counts, world, r) for r in range(world)]  # deterministic
    with pytest.raises(ValueError):
        shard_scenes(counts, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, T, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = scenes.make("rects2d", n_scenes=5, n_min=200, n_max=600)
    mine = shard_scenes(base["desc"]["n_particles"], world, rank)
    res = oracle.simulate(scenes.oracle_view(subset(base, mine)), T)
    gathered = [None] * world
    dist.all_gather_object(gathered, {i: r for i, r in zip(mine, res)})
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        q.put((merged, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_run_equals_single_process():
    T = 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, T, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == 2.0  # max over ranks
    base = scenes.make("rects2d", n_scenes=5, n_min=200, n_max=600)
    single = oracle.simulate(scenes.oracle_view(base), T)
    assert sorted(merged) == list(range(5))
    for i in range(5):
        np.testing.assert_array_equal(merged[i], single[i])  # bitwise


def _failing_worker(rank, world, port, q):
    store = dist.TCPStore("127.0.0.1", port, world, is_master=(rank == 0),
                          timeout=__import__("datetime").timedelta(seconds=30))
    if rank == 1:
        raise RuntimeError("simulated rank failure before its shard is reported")
    base = scenes.make("rects2d", n_scenes=3, n_min=200, n_max=400)
    mine = shard_scenes(base["desc"]["n_particles"], world, rank)
    res = oracle.simulate(scenes.oracle_view(subset(base, mine)), 2)
    try:
        collect_shards(store, rank, world, {i: r for i, r in zip(mine, res)}, timeout_s=5.0)
        q.put(("no failure detected", None))
    except RankFailure as e:
        q.put(("detected", e.missing))


def test_failed_rank_is_detected_without_a_hang():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    status, missing = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert status == "detected" and missing == [1]
    assert procs[0].exitcode == 0 and procs[1].exitcode != 0


def test_collect_shards_returns_every_rank():
    store = dist.HashStore()
    assert collect_shards(store, 1, 2, {"b": 2}) is None
    got = collect_shards(store, 0, 2, {"a": 1}, timeout_s=5.0)
    assert got == {0: {"a": 1}, 1: {"b": 2}}


def _grad_worker(rank, world, port, T, q):
    """The benchmark's --shard split of one batch: each rank runs forward, loss and backward
    on its scenes and publishes losses and gradients through the store."""
    store = dist.TCPStore("127.0.0.1", port, world, is_master=(rank == 0),
                          timeout=__import__("datetime").timedelta(seconds=60))
    base = scenes.make("robots3d", n_scenes=3, dims=(8, 6, 6), n_grid=32)
    mine = shard_scenes(base["desc"]["n_particles"], world, rank)
    r = oracle.loss_and_grad(scenes.oracle_view(subset(base, mine)), T)
    off = np.concatenate([[0], np.cumsum(subset(base, mine)["desc"]["n_particles"])])
    per = {}
    for j, i in enumerate(mine):
        sl = slice(int(off[j]), int(off[j + 1]))
        per[i] = dict(loss=r["losses"][j], gx0=r["gx0"][:, sl], gv0=r["gv0"][:, sl],
                      gE=r["gE"][sl], gw=r["gw"][j])
    got = collect_shards(store, rank, world, per, timeout_s=120.0, tag="grad")
    if rank == 0:
        merged = {}
        for v in got.values():
            merged.update(v)
        q.put(merged)


def test_two_rank_sharded_gradients_equal_single_process():
    T = 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, T, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    base = scenes.make("robots3d", n_scenes=3, dims=(8, 6, 6), n_grid=32)
    assert sorted(merged) == [0, 1, 2]
    assert sorted(shard_scenes(base["desc"]["n_particles"], 2, 0) +
                  shard_scenes(base["desc"]["n_particles"], 2, 1)) == [0, 1, 2]
    single = oracle.loss_and_grad(scenes.oracle_view(base), T)
    off = np.concatenate([[0], np.cumsum(base["desc"]["n_particles"])])
    for i in range(3):
        sl = slice(int(off[i]), int(off[i + 1]))
        assert merged[i]["loss"] == single["losses"][i]  # bitwise
        for k in ("gx0", "gv0"):
            np.testing.assert_array_equal(merged[i][k], single[k][:, sl])
        np.testing.assert_array_equal(merged[i]["gE"], single["gE"][sl])
        np.testing.assert_array_equal(merged[i]["gw"], single["gw"][i])
