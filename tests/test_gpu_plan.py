"""Batch plans: graph-replayed builds and autotuned search options vs the oracle (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1803_09835_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def _stations(lengths, seed_shift=0, **over):
    ws = [synth.scaled("c2", n, station=s + seed_shift, **over) for s, n in enumerate(lengths)]
    return ws, [synth.generate(w, ld=((w.K + 7) // 8) * 8) for w in ws]


def _want(p, w, a):
    keys = oracle.keys(p, np.ascontiguousarray(a[:, :w.K]))
    return oracle.search(p, keys, oracle.drop(p, keys))


def _eq(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_plan_replays_match_oracle_on_refilled_input():
    from paper_1803_09835_gb300 import Searcher
    lengths = [4000, 1500, 7000, 2500]
    st = torch.cuda.Stream()
    s = Searcher(synth.scaled("c2", 1000, D=2048, K=100, b=30).params(), timing=1)
    buf = None
    plan = None
    for rnd in range(3):
        ws, idx = _stations(lengths, seed_shift=10 * rnd, D=2048, K=100, b=30)
        host = torch.from_numpy(np.concatenate(idx))
        if buf is None:
            buf = host.cuda()
            torch.cuda.synchronize()
            plan = s.plan(buf, lengths, st)
        else:
            buf.copy_(host)
            torch.cuda.synchronize()
        res = plan.run()
        for x, (w, a) in enumerate(zip(ws, idx)):
            assert _eq(res[x].numpy(), _want(w.params(), w, a)), f"run {rnd} station {x}"
            res[x].free()
        info = plan.info()
        assert info["tuned"] and len(info["tried"]) == 7 and info["graph_kernels"] > 10
        assert info["best"]["ms"] == min(t["ms"] for t in info["tried"])
        assert info["build_ms"] > 0
    plan.close()
    s.close()


def test_plan_keeps_context_options_and_matches_detect_batch():
    from paper_1803_09835_gb300 import Searcher
    lengths = [3000, 3000]
    ws, idx = _stations(lengths, D=2048, K=100, b=20)
    s = Searcher(ws[0].params(), large_min=16)
    st = torch.cuda.Stream()
    buf = torch.from_numpy(np.concatenate(idx)).cuda()
    torch.cuda.synchronize()
    plan = s.plan(buf, lengths, st)
    a = [r.numpy() for r in plan.run()]
    b = [r.numpy() for r in plan.run()]
    with torch.cuda.stream(st):
        c = [r.numpy() for r in s.detect_batch(buf, lengths, stream=st)]
    for x in range(2):
        assert _eq(a[x], b[x]) and _eq(a[x], c[x])
    # the context still searches with its own dense-group threshold of 16
    s.detect(buf)
    s2 = Searcher(ws[0].params(), large_min=16)
    s2.detect(buf)
    assert s.stats()["n_groups"] == s2.stats()["n_groups"]
    s2.close()
    plan.close()
    s.close()


def test_plan_rejects_bad_shapes():
    from paper_1803_09835_gb300 import FastError, Searcher
    ws, idx = _stations([1000], D=2048, K=100, b=20)
    s = Searcher(ws[0].params())
    buf = torch.from_numpy(idx[0]).cuda()
    st = torch.cuda.Stream()
    with pytest.raises(FastError):
        s.plan(buf, [0, 0], st)
    with pytest.raises(FastError):
        s.plan(buf, [], st)
    s.close()
