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
