"""Batched multi-station search (one pass over uneven stations) vs per-station results (GPU)."""
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


def _stations(lengths, **over):
    ws = [synth.scaled("c2", n, station=s, **over) for s, n in enumerate(lengths)]
    return ws, [synth.generate(w, ld=((w.K + 7) // 8) * 8) for w in ws]


def _eq(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("opts", [{}, {"large_min": 16}, {"vote_map": 1}])
def test_uneven_stations_equal_single_station_runs(opts):
    from paper_1803_09835_gb300 import Searcher
    lengths = [s * 1500 for s in range(1, 13)]
    ws, idx = _stations(lengths, D=2048, K=100, b=30)
    p = ws[0].params()
    s = Searcher(p, **opts)
    batch = s.detect_batch(torch.from_numpy(np.concatenate(idx)).cuda(), lengths)
    for x, (w, a) in enumerate(zip(ws, idx)):
        keys = oracle.keys(p, np.ascontiguousarray(a[:, :w.K]))
        want = oracle.search(p, keys, oracle.drop(p, keys))
        got = batch[x].numpy()
        assert _eq(got, want), f"station {x}"
        alone = s.detect(torch.from_numpy(a).cuda())
        assert _eq(alone.numpy(), got)
        alone.free()
    for r in batch:
        r.free()
    s.close()


def test_batch_thresholds_are_per_station():
    # with the automatic dense threshold every station of a batch keeps its
    # own: station a's buckets of 520..775 windows are dense alone, and stay
    # dense next to station b, whose largest bucket (~15,500) would lift one
    # batch-wide threshold above them
    from dataclasses import replace

    from paper_1803_09835_gb300 import Searcher
    a = replace(synth.scaled("c2", 40_000, station=0, D=2048, K=100, b=30, occ_num=0), periods=(40,))
    b = replace(synth.scaled("c2", 40_000, station=1, D=2048, K=100, b=30, occ_num=0), periods=(2,))
    ia, ib = (synth.generate(w, ld=104) for w in (a, b))
    s = Searcher(a.params())
    keys = ("n_dense_pairs", "n_emissions", "n_groups", "n_detections")
    alone = []
    for x in (ia, ib):
        r = s.detect(torch.from_numpy(x).cuda())
        st = s.stats()
        alone.append((r.numpy(), {k: st[k] for k in keys}, st["large_min"]))
        r.free()
    assert alone[0][1]["n_groups"] > 0 and alone[1][1]["n_groups"] > 0
    batch = s.detect_batch(torch.from_numpy(np.concatenate([ia, ib])).cuda(), [a.N, b.N])
    st = s.stats()
    for x in range(2):
        assert _eq(batch[x].numpy(), alone[x][0]), f"station {x}"
        batch[x].free()
    for k in keys:
        assert st[k] == alone[0][1][k] + alone[1][1][k], k
    assert st["large_min"] == max(alone[0][2], alone[1][2])
    s.close()


def test_equal_keys_across_a_station_boundary():
    # station 1 repeats station 0 window for window: the last keys of one
    # station equal the first keys of the next, and buckets must not merge
    from paper_1803_09835_gb300 import Searcher
    ws, idx = _stations([3000], D=2048, K=100, b=20)
    a = idx[0]
    p = ws[0].params()
    s = Searcher(p)
    batch = s.detect_batch(torch.from_numpy(np.concatenate([a, a, a[:1000]])).cuda(), [3000, 3000, 1000])
    keys = oracle.keys(p, np.ascontiguousarray(a[:, :100]))
    want = oracle.search(p, keys, oracle.drop(p, keys))
    assert _eq(batch[0].numpy(), want) and _eq(batch[1].numpy(), want)
    k2 = np.ascontiguousarray(keys[:, :1000])
    assert _eq(batch[2].numpy(), oracle.search(p, k2, oracle.drop(p, k2)))
    s.close()


def test_batch_of_one_and_empty_stations():
    from paper_1803_09835_gb300 import Searcher
    ws, idx = _stations([2500], D=2048, K=100, b=20)
    p = ws[0].params()
    s = Searcher(p)
    a = torch.from_numpy(idx[0]).cuda()
    one = s.detect_batch(a, [2500])[0].numpy()
    ref = s.detect(a).numpy()
    assert _eq(one, ref)
    parts = s.detect_batch(a, [0, 2500, 0])
    assert parts[0].M == 0 and parts[2].M == 0 and _eq(parts[1].numpy(), ref)
    s.close()


@pytest.mark.slow
def test_c2_four_and_three_month_batch_full_size():
    """Two stations of the 12-station workload at full size (4 and 3 months,
    18,144,000 windows) in one batch: each station's drop count equals the
    oracle's, its list is sorted, unique and within the rules, and sampled
    rows equal the oracle's rows."""
    from paper_1803_09835_gb300 import Searcher
    ws = [synth.workload("c2", station=3), synth.workload("c2", station=2)]
    idx = [synth.generate(w, ld=400) for w in ws]
    p = ws[0].params()
    s = Searcher(dict(p, table_group=10))
    res = s.detect_batch(torch.from_numpy(np.concatenate(idx)).cuda(), [w.N for w in ws])
    got = [r.numpy() for r in res]
    for r in res:
        r.free()
    s.close()
    torch.cuda.empty_cache()
    rng = np.random.default_rng(7)
    for (gi, gj, gv), w, a in zip(got, ws, idx):
        assert len(gi) > 10**8
        assert np.all(gi < gj) and np.all(gj.astype(np.int64) - gi > p["excl"]) and np.all(gv >= p["v"])
        key = (gi.astype(np.uint64) << np.uint64(32)) | gj
        assert np.all(key[1:] > key[:-1])
        del key
        keys = oracle.keys(p, a)
        drop = oracle.drop(p, keys)
        assert not drop[gi].any() and not drop[gj].any()
        rows = np.concatenate([rng.choice(np.unique(gi[::9973]), 6, replace=False), rng.integers(0, w.N, 4)])
        starts, ends = np.searchsorted(gi, rows), np.searchsorted(gi, rows, side="right")
        for row, lo, hi in zip(rows, starts, ends):
            wj, wv = oracle.search_row(p, keys, drop, int(row))
            assert np.array_equal(gj[lo:hi], wj) and np.array_equal(gv[lo:hi], wv), f"row {row}"
        del keys
