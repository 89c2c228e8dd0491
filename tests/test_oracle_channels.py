"""Pins of the oracle's channel level (§7.1 "Channel Level", computed by the
sort-merge-reduce of §7.2): the channels' (i, j, votes) lists of one station
summed per pair and thresholded again, output in (dt, idx1) order (CPU only).

The oracle follows the paper's sort / merge / reduce phases; the pins check
it against the paper's own "naive" alternative (one hash map of the summed
entries), against invariants of the definition, and on detection lists of a
synthetic station searched three times with independent hash families."""
import numpy as np
import pytest

import oracle
import synth


def _dict_merge(lists, thr):
    """The hash-map form §7.2 names: accumulate every channel's entries, keep
    the sums >= thr, order by (dt = j - i, idx1 = i)."""
    acc = {}
    for i, j, v in lists:
        for a, b, c in zip(i.tolist(), j.tolist(), v.tolist()):
            acc[(a, b)] = acc.get((a, b), 0) + c
    kept = sorted(((b - a, a, s) for (a, b), s in acc.items() if s >= thr))
    return (np.array([a for _, a, _ in kept], np.uint32), np.array([dt + a for dt, a, _ in kept], np.uint32),
            np.array([s for _, _, s in kept], np.uint16))


def _random_lists(rng, nch, n, span, maxv=255):
    out = []
    for _ in range(nch):
        i = rng.integers(0, span, n)
        j = i + rng.integers(1, 40, n)
        pairs = sorted(set(zip(i.tolist(), j.tolist())))  # a detection list holds each pair once
        i = np.array([a for a, _ in pairs], np.uint32)
        j = np.array([b for _, b in pairs], np.uint32)
        v = rng.integers(1, maxv + 1, len(pairs)).astype(np.uint8)
        out.append((i, j, v))
    return out


def _eq(a, b):
    assert all(np.array_equal(x, y) for x, y in zip(a, b)), (a, b)


@pytest.mark.parametrize("seed,nch,thr", [(1, 3, 5), (2, 3, 1), (3, 2, 300), (4, 1, 0), (5, 5, 200)])
def test_matches_the_hash_map_form(seed, nch, thr):
    rng = np.random.default_rng(seed)
    lists = _random_lists(rng, nch, 2000, 300)  # dense enough that channels share many pairs
    _eq(oracle.channel_merge(lists, thr), _dict_merge(lists, thr))


def test_channel_order_does_not_matter():
    rng = np.random.default_rng(7)
    lists = _random_lists(rng, 3, 1500, 200)
    ref = oracle.channel_merge(lists, 6)
    for perm in ((1, 0, 2), (2, 1, 0), (2, 0, 1)):
        _eq(oracle.channel_merge([lists[k] for k in perm], 6), ref)


def test_sums_are_conserved_and_thresholds_nest():
    rng = np.random.default_rng(11)
    lists = _random_lists(rng, 3, 1000, 150)
    i0, j0, s0 = oracle.channel_merge(lists, 0)
    assert int(s0.astype(np.int64).sum()) == sum(int(v.astype(np.int64).sum()) for _, _, v in lists)
    assert len(i0) == len({p for i, j, _ in lists for p in zip(i.tolist(), j.tolist())})
    prev = None
    for thr in (0, 2, 50, 256, 500, 766):
        got = oracle.channel_merge(lists, thr)
        keep = s0 >= thr
        _eq(got, (i0[keep], j0[keep], s0[keep]))  # exactly the sums >= thr, order kept
        if prev is not None:
            assert len(got[0]) <= len(prev[0])
        prev = got
    assert len(oracle.channel_merge(lists, 766)[0]) == 0  # three channels sum to at most 765


def test_one_channel_is_its_list_in_diagonal_order():
    rng = np.random.default_rng(13)
    (i, j, v), = _random_lists(rng, 1, 800, 100)
    gi, gj, gs = oracle.channel_merge([(i, j, v)], 0)
    order = np.lexsort((i, j - i))
    _eq((gi, gj, gs), (i[order], j[order], v[order].astype(np.uint16)))


def test_empty_inputs():
    e = (np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    for lists in ([], [e], [e, e, e]):
        gi, gj, gs = oracle.channel_merge(lists, 1)
        assert len(gi) == len(gj) == len(gs) == 0


def test_three_searches_of_one_station():
    # three independent hash families over one synthetic station stand in for
    # its three channels: repeated templates are found in all of them, chance
    # collisions mostly in one; the merged list keeps a pair when the summed
    # votes reach the raised threshold
    w = synth.scaled("c0", 4096)
    idx = synth.generate(w)
    lists = []
    for k in range(3):
        p = dict(w.params(), seed=w.params()["seed"] + 1000 * k)
        keys = oracle.keys(p, idx)
        lists.append(oracle.search(p, keys, oracle.drop(p, keys)))
    assert all(len(l[0]) > 0 for l in lists)
    thr = 3 * w.params()["v"]
    got = oracle.channel_merge(lists, thr)
    _eq(got, _dict_merge(lists, thr))
    assert 0 < len(got[0]) <= len(_dict_merge(lists, 0)[0])
