"""Alignment steps on the GPU vs the oracle (§7.1, §7.2).

Channel level: the channels' detection lists summed per pair and thresholded
again, in (dt, idx1) order -- element-wise equal to the oracle's
sort-merge-reduce.  Station level: thin diagonal clusters with their summary
statistics -- the same set of clusters as the oracle, in (dt_min, idx1_min)
order.
"""
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


def _searcher(p=None, **opts):
    from paper_1803_09835_gb300 import Searcher
    p = p or dict(D=2048, K=100, b=16, r=4, kind=0, seed=1, v=2, excl=5, occ_num=0, occ_den=1)
    return Searcher(p, **opts)


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


class _List:
    """A detection list uploaded as device tensors (what Searcher.channel_merge reads)."""

    def __init__(self, i, j, v):
        self.M = len(i)
        self.i = _dev(i.astype(np.uint32), np.int32)
        self.j = _dev(j.astype(np.uint32), np.int32)
        self.votes = _dev(v.astype(np.uint8), np.uint8)


def _eq(a, b):
    assert len(a[0]) == len(b[0]), (len(a[0]), len(b[0]))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def _random_lists(rng, nch, n, span, maxv=255):
    out = []
    for _ in range(nch):
        i = rng.integers(0, span, n)
        j = i + rng.integers(1, 40, n)
        pairs = sorted(set(zip(i.tolist(), j.tolist())))
        i = np.array([a for a, _ in pairs], np.uint32)
        j = np.array([b for _, b in pairs], np.uint32)
        out.append((i, j, rng.integers(1, maxv + 1, len(pairs)).astype(np.uint8)))
    return out


@pytest.mark.parametrize("seed,nch,thr", [(1, 3, 5), (2, 3, 1), (3, 2, 300), (4, 1, 0), (5, 5, 200), (6, 8, 700)])
def test_channel_merge_random_lists(seed, nch, thr):
    rng = np.random.default_rng(seed)
    lists = _random_lists(rng, nch, 20_000, 3000)
    s = _searcher()
    m = s.channel_merge([_List(*l) for l in lists], N=3100, thr=thr)
    _eq(m.numpy(), oracle.channel_merge(lists, thr))
    m.free()
    s.close()


def test_channel_merge_empty_and_bad_input():
    from paper_1803_09835_gb300 import FastError, _lib
    s = _searcher()
    e = (np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    rng = np.random.default_rng(3)
    one = _random_lists(rng, 1, 500, 100)[0]
    for lists in ([e], [e, e, e], [e, one, e]):
        m = s.channel_merge([_List(*l) for l in lists], N=200, thr=1)
        _eq(m.numpy(), oracle.channel_merge(lists, 1))
        m.free()
    for bad in ((np.array([5], np.uint32), np.array([5], np.uint32)),      # j == i
                (np.array([5], np.uint32), np.array([250], np.uint32))):   # j >= N
        with pytest.raises(FastError) as ex:
            s.channel_merge([_List(bad[0], bad[1], np.ones(1, np.uint8))], N=200, thr=1)
        assert ex.value.status == _lib.FAST_EINVAL
    # the context stays usable
    m = s.channel_merge([_List(*one)], N=200, thr=0)
    _eq(m.numpy(), oracle.channel_merge([one], 0))
    s.close()


def _three_channels(n):
    # three independent hash families over one synthetic station stand in for
    # its three channels (each searched on the GPU and by the oracle)
    w = synth.scaled("c1", n)
    idx = synth.generate(w, ld=400)
    ps = [dict(w.params(), seed=w.params()["seed"] + 1000 * k) for k in range(3)]
    gpu, want, ctxs = [], [], []
    for p in ps:
        s = _searcher(p)
        ctxs.append(s)  # a result may not outlive the context that made it
        gpu.append(s.detect(torch.from_numpy(idx).cuda()))
        keys = oracle.keys(p, idx)
        want.append(oracle.search(p, keys, oracle.drop(p, keys)))
        _eq(gpu[-1].numpy(), want[-1])
    return w, gpu, want, ctxs


def test_channel_merge_then_station_clusters_on_three_searches():
    w, gpu, want, ctxs = _three_channels(60_000)
    assert all(len(x[0]) > 0 for x in want)
    s = _searcher(w.params())
    for thr in (0, w.v + 1, 3 * w.v):
        m = s.channel_merge(gpu, N=w.N, thr=thr)
        ref = oracle.channel_merge(want, thr)
        assert len(ref[0]) > 0
        _eq(m.numpy(), ref)
        for gap, width, min_n in ((1, 1, 1), (5, 3, 2), (40, 6, 3)):
            c = s.station_clusters(m, gap=gap, width=width, min_n=min_n)
            _clusters_eq(c.numpy(), oracle.station_clusters(*ref, gap=gap, width=width, min_n=min_n))
            c.free()
        m.free()
    for r in gpu:
        r.free()
    for c in ctxs:
        c.close()
    s.close()


def _order(i, j, s):
    o = np.lexsort((i, j - i))
    return i[o], j[o], s[o]


def _clusters_eq(got, want):
    assert got.shape == want.shape, (got.shape, want.shape)
    if len(got):
        key = got[:, 0] * (1 << 32) + got[:, 2]
        assert np.all(np.diff(key) >= 0)  # (dt_min, idx1_min) order
    lg, lw = np.lexsort(got.T[::-1]), np.lexsort(want.T[::-1])
    assert np.array_equal(got[lg], want[lw])


def _station_list(rng, n, span, dts):
    i = rng.integers(0, span, n).astype(np.uint32)
    j = (i + rng.integers(1, dts, n)).astype(np.uint32)
    pairs = sorted(set(zip(i.tolist(), j.tolist())))
    i = np.array([a for a, _ in pairs], np.uint32)
    j = np.array([b for _, b in pairs], np.uint32)
    s = rng.integers(1, 300, len(pairs)).astype(np.uint16)
    return _order(i, j, s)


def _clusters(s, i, j, sim, **kw):
    c = s.station_clusters((_dev(i, np.int32), _dev(j, np.int32), _dev(sim, np.int16)), **kw)
    out = c.numpy()
    c.free()
    return out


@pytest.mark.parametrize("seed,n,span,dts,gap,width,min_n", [
    (1, 3000, 2000, 6, 1, 1, 1), (2, 3000, 2000, 6, 3, 2, 1), (3, 40_000, 30_000, 12, 8, 3, 2),
    (4, 40_000, 30_000, 12, 8, 6, 5), (5, 200_000, 50_000, 30, 4, 4, 1), (6, 200_000, 400_000, 200, 40, 2, 3)])
def test_station_clusters_random_lists(seed, n, span, dts, gap, width, min_n):
    rng = np.random.default_rng(seed)
    i, j, sim = _station_list(rng, n, span, dts)
    s = _searcher()
    _clusters_eq(_clusters(s, i, j, sim, gap=gap, width=width, min_n=min_n),
                 oracle.station_clusters(i, j, sim, gap=gap, width=width, min_n=min_n))
    s.close()


def test_station_clusters_long_staircases_need_many_rounds():
    # near runs chained over hundreds of adjacent diagonals: the width limit
    # restarts clusters periodically along each chain, and every run's choice
    # waits for the diagonal below
    pts = []
    for band in range(5):
        t0, d0 = 10_000 * band, 50 + 1000 * band
        for k in range(300 + 50 * band):
            for x in range(3):
                pts.append((t0 + k + x, t0 + k + x + d0 + k))
    i = np.array([a for a, _ in pts], np.uint32)
    j = np.array([b for _, b in pts], np.uint32)
    sim = np.arange(len(i), dtype=np.uint16) % 7 + 1
    i, j, sim = _order(i, j, sim)
    s = _searcher()
    for width in (1, 2, 3, 7):
        _clusters_eq(_clusters(s, i, j, sim, gap=3, width=width, min_n=1),
                     oracle.station_clusters(i, j, sim, gap=3, width=width, min_n=1))
    s.close()


def test_station_clusters_worked_staircase_and_bad_input():
    from paper_1803_09835_gb300 import FastError, _lib
    i = np.arange(1000, 1006, dtype=np.uint32)
    j = (i + 100 + np.arange(6)).astype(np.uint32)
    sim = np.ones(6, np.uint16)
    i, j, sim = _order(i, j, sim)
    s = _searcher()
    assert _clusters(s, i, j, sim, gap=3, width=6, min_n=1).tolist() == [[100, 105, 1000, 1005, 6, 6]]
    assert _clusters(s, i, j, sim, gap=3, width=3, min_n=1).tolist() == [[100, 102, 1000, 1002, 3, 3],
                                                                          [103, 105, 1003, 1005, 3, 3]]
    assert _clusters(s, i[:0], j[:0], sim[:0], gap=3, width=3, min_n=1).shape == (0, 6)
    # the search's own (i, j) order is not (dt, idx1) order
    bi, bj = np.array([5, 5, 6], np.uint32), np.array([20, 30, 21], np.uint32)
    with pytest.raises(FastError) as ex:
        _clusters(s, bi, bj, np.ones(3, np.uint16), gap=3, width=2, min_n=1)
    assert ex.value.status == _lib.FAST_EINVAL
    with pytest.raises(FastError):
        _clusters(s, i, j, sim, gap=0, width=2, min_n=1)
    s.close()
