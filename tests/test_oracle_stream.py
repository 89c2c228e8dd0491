"""Pins of the oracle's streaming replay (CPU only)."""
import numpy as np

import oracle
import synth


def _wl(n, **over):
    return synth.scaled("c3", n, D=2048, K=100, b=24, **over)


def test_batches_partition_the_plain_search_without_filter():
    # With no history and no filter, the requests' pairs (j in the batch) over
    # consecutive batches are exactly the plain search's pairs.
    w = _wl(2400, occ_num=0)
    idx = synth.generate(w)
    p = w.params()
    keys = oracle.keys(p, idx)
    want = oracle.search(p, keys, None)
    cuts = [0, 300, 700, 1500, 2400]
    got = [[], [], []]
    for a, b in zip(cuts[:-1], cuts[1:]):
        i, j, v = oracle.stream_query(p, np.ascontiguousarray(keys[:, :b]), 0, a, None)
        for g, x in zip(got, (i, j, v)):
            g.append(x)
    got = [np.concatenate(g) for g in got]
    order = np.lexsort((got[1], got[0]))
    for g, x in zip(got, want):
        assert np.array_equal(g[order], x)


def test_copies_of_dropped_history_windows_are_dropped():
    w = _wl(3000)
    idx = synth.generate(w)
    p = w.params()
    n0 = 2500
    hk = oracle.keys(p, idx[:n0])
    hd = oracle.drop(p, hk)
    dropped = np.nonzero(hd)[0]
    assert len(dropped) > 10
    batch = np.concatenate([idx[n0:n0 + 50], idx[dropped[:20]]])
    allidx = np.concatenate([idx[:n0], batch])
    keys = oracle.keys(p, allidx)
    i, j, v = oracle.stream_query(p, keys, n0, n0, hd)
    copies = set(range(n0 + 50, n0 + 70))
    assert not copies & set(j.tolist()) and not copies & set(i.tolist())
    assert not set(dropped.tolist()) & set(i.tolist())
