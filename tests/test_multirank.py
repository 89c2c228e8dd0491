"""The N > 1 bench path on CPU ranks (gloo, world size 2): one station per
rank, no data-path collective, max-over-ranks timing, weak-scaling value."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.station_workload("c1", rank, n=3000)
        idx = synth.generate(w, ld=w.K)
        p = w.params()
        ms, out = bench.timed_steps(lambda: oracle.run(p, idx), steps=2, warmup=1, dist=dist)
        ms_max = bench.max_over_ranks(ms, dist)
        every = [None] * world
        dist.all_gather_object(every, ms)
        value = bench.weak_value([w.N] * world, ms_max)
        q.put(dict(rank=rank, ms=ms, ms_max=ms_max, every=every, value=value, seed=w.seed,
                   M=len(out[0]), N=w.N))
    finally:
        dist.destroy_process_group()


def test_two_ranks_one_station_each_max_timing():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=300)
        res[r["rank"]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = res[0], res[1]
    assert a["seed"] != b["seed"]                      # each rank its own station
    assert a["ms_max"] == b["ms_max"] == pytest.approx(max(a["every"]))
    assert a["ms_max"] >= a["ms"] and a["ms_max"] >= b["ms"]
    assert a["value"] == pytest.approx((a["N"] + b["N"]) / (a["ms_max"] / 1000))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    ms, out = bench.timed_steps(lambda: calls.append(1) or len(calls), steps=3, warmup=2)
    assert len(calls) == 5 and out == 5 and ms >= 0
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.weak_value([1000, 3000], 2.0) == pytest.approx(2e6)
    w0, w1 = bench.station_workload("c1", 0, 500), bench.station_workload("c1", 1, 500)
    assert w0.N == w1.N == 500 and w0.seed != w1.seed


def _split_main(rank, world, port, q):
    """One station split by table group over CPU ranks: each rank's partial
    votes and heavy counts come from the oracle over its own tables; the
    product's shard module all-reduces the heavy counts, exchanges the
    partial votes by owner and reduces them."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1803_09835_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.scaled("c1", 8000)
        idx = synth.generate(w, ld=w.K)
        p = w.params()
        keys = oracle.keys(p, idx)
        t0, t1 = shard.table_range(p["b"], rank, world)
        mine = np.ascontiguousarray(keys[t0:t1])
        sub = dict(p, b=t1 - t0, v=1)
        _, heavy = oracle.drop(sub, mine, heavy_cnt=True)
        drop = shard.drop_from_heavy(shard.all_reduce_counts(dist, heavy), p["b"])
        pi, pj, pv = oracle.search(sub, mine, drop)  # pairs sharing >= 1 of this rank's tables
        part = shard.reduce_owned(*shard.exchange(dist, pi, pj, pv), p["v"])
        owned = shard.owner(part[0], part[1], world)
        merged = shard.gather_sorted(dist, part)
        res = dict(rank=rank, tables=(t0, t1), partial=len(pi), owned_ok=bool(np.all(owned == rank)))
        if rank == 0:
            full_drop = oracle.drop(p, keys)
            want = oracle.search(p, keys, full_drop)
            res.update(same_drop=bool(np.array_equal(drop, full_drop)), n_drop=int(full_drop.sum()),
                       same=all(np.array_equal(a, b) for a, b in zip(merged, want)), M=len(want[0]))
        q.put(res)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_table_group_split_equals_the_single_rank_search(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=300)
        res[r["rank"]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res[r]["tables"] for r in res) == [((100 * k) // world, (100 * (k + 1)) // world)
                                                     for k in range(world)]
    assert all(res[r]["owned_ok"] and res[r]["partial"] > 0 for r in res)
    assert res[0]["same_drop"] and res[0]["n_drop"] > 0
    assert res[0]["same"] and res[0]["M"] > 0


def test_shard_helpers_single_process():
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_1803_09835_gb300 import shard
    assert [shard.table_range(100, r, 3) for r in range(3)] == [(0, 33), (33, 66), (66, 100)]
    i = np.array([5, 5, 7, 5], np.uint32)
    j = np.array([9, 9, 20, 30], np.uint32)
    v = np.array([2, 3, 4, 1], np.uint32)
    ri, rj, rv = shard.reduce_owned(i, j, v, 3)
    assert list(zip(ri.tolist(), rj.tolist(), rv.tolist())) == [(5, 9, 5), (7, 20, 4)]
    o = shard.owner(np.arange(1000, dtype=np.uint32), np.arange(1000, dtype=np.uint32) + 7, 4)
    assert set(o.tolist()) == {0, 1, 2, 3} and np.array_equal(o, shard.owner(np.arange(1000, dtype=np.uint32),
                                                                              np.arange(1000, dtype=np.uint32) + 7, 4))
    assert shard.drop_from_heavy(np.array([0, 50, 51]), 100).tolist() == [0, 0, 1]
