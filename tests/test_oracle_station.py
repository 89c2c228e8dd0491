"""Pins of the oracle's station level (§7.1 "Station Level", §7.2 "Station"):
thin diagonal clusters of a (dt, idx1)-ordered similarity list, summarised
by bounding box, entry count and summed similarity (CPU only)."""
import numpy as np
import pytest

import oracle


def _order(i, j, s):
    o = np.lexsort((i, j - i))
    return i[o], j[o], s[o]


def _runs(i, j, s, gap):
    """Direct definition of the per-diagonal sequences: consecutive entries of
    one diagonal whose idx1 differ by less than gap."""
    out = []
    for k in range(len(i)):
        dt = int(j[k] - i[k])
        if out and out[-1][0] == dt and int(i[k]) - out[-1][3] < gap:
            c = out[-1]
            out[-1] = (dt, dt, c[2], int(i[k]), c[4] + 1, c[5] + int(s[k]))
        else:
            out.append((dt, dt, int(i[k]), int(i[k]), 1, int(s[k])))
    return np.array(sorted(out), np.int64).reshape(-1, 6)


def _random_list(rng, n, span, dts):
    i = rng.integers(0, span, n).astype(np.uint32)
    j = (i + rng.integers(1, dts, n)).astype(np.uint32)
    pairs = sorted(set(zip(i.tolist(), j.tolist())))
    i = np.array([a for a, _ in pairs], np.uint32)
    j = np.array([b for _, b in pairs], np.uint32)
    s = rng.integers(1, 300, len(pairs)).astype(np.uint16)
    return _order(i, j, s)


@pytest.mark.parametrize("seed,gap", [(1, 1), (2, 3), (3, 10), (4, 40)])
def test_runs_along_one_diagonal(seed, gap):
    rng = np.random.default_rng(seed)
    i, j, s = _random_list(rng, 3000, 2000, 6)  # few diagonals, dense runs
    got = oracle.station_clusters(i, j, s, gap=gap, width=1, min_n=1)
    assert np.array_equal(got, _runs(i, j, s, gap))


def test_conservation_width_and_pruning():
    rng = np.random.default_rng(5)
    i, j, s = _random_list(rng, 4000, 3000, 12)
    for width in (1, 2, 3, 6):
        all_ = oracle.station_clusters(i, j, s, gap=8, width=width, min_n=1)
        assert all_[:, 4].sum() == len(i) and all_[:, 5].sum() == int(s.astype(np.int64).sum())
        assert (all_[:, 1] - all_[:, 0] + 1 <= width).all() and (all_[:, 2] <= all_[:, 3]).all()
        for min_n in (2, 5, 30):
            assert np.array_equal(oracle.station_clusters(i, j, s, gap=8, width=width, min_n=min_n),
                                  all_[all_[:, 4] >= min_n])
    # merging across diagonals only joins runs; a larger gap only joins runs
    runs = len(oracle.station_clusters(i, j, s, gap=8, width=1, min_n=1))
    assert all(len(oracle.station_clusters(i, j, s, gap=8, width=w, min_n=1)) <= runs for w in (2, 4, 8))
    counts = [len(oracle.station_clusters(i, j, s, gap=g, width=1, min_n=1)) for g in (1, 4, 16, 64)]
    assert counts == sorted(counts, reverse=True)


def test_every_entry_inside_its_box():
    rng = np.random.default_rng(9)
    i, j, s = _random_list(rng, 2000, 4000, 8)
    boxes = oracle.station_clusters(i, j, s, gap=6, width=3, min_n=1)
    dt = (j - i).astype(np.int64)
    inside = np.zeros(len(i), np.int64)
    for b in boxes:
        inside += (dt >= b[0]) & (dt <= b[1]) & (i >= b[2]) & (i <= b[3])
    assert (inside >= 1).all()  # boxes may overlap, but each entry lies in one


def test_events_are_recovered_and_isolated_matches_pruned():
    # three reoccurring events: thin diagonals of 20..40 matches (one window
    # apart, some skipped), drifting over up to three adjacent diagonals; plus
    # isolated chance matches far from them
    rng = np.random.default_rng(21)
    pts, events = [], []
    for dt0, t0 in ((300, 1000), (5000, 20000), (86400, 500)):
        length = int(rng.integers(20, 41))
        ev = []
        for k in range(length):
            if rng.random() < 0.2:
                continue
            dt = dt0 + (k * 3) // length  # drifts by at most two diagonals
            ev.append((t0 + k, t0 + k + dt, int(rng.integers(4, 20))))
        pts += ev
        dts = [b - a for a, b, _ in ev]
        events.append((min(dts), max(dts), min(a for a, _, _ in ev), max(a for a, _, _ in ev)))
    for _ in range(50):
        a = int(rng.integers(100_000, 200_000))
        pts.append((a, a + int(rng.integers(11, 50_000)), 4))
    i, j, s = (np.array(x, t) for x, t in zip(zip(*pts), (np.uint32, np.uint32, np.uint16)))
    i, j, s = _order(i, j, s)
    got = oracle.station_clusters(i, j, s, gap=5, width=3, min_n=3)
    assert sorted(map(tuple, got[:, :4].tolist())) == sorted(map(tuple, events))


def test_width_limit_splits_a_wide_staircase():
    # one match per diagonal over six adjacent diagonals, one window apart
    i = np.arange(1000, 1006, dtype=np.uint32)
    j = (i + 100 + np.arange(6)).astype(np.uint32)
    s = np.ones(6, np.uint16)
    i, j, s = _order(i, j, s)
    one = oracle.station_clusters(i, j, s, gap=3, width=6, min_n=1)
    assert one.tolist() == [[100, 105, 1000, 1005, 6, 6]]
    two = oracle.station_clusters(i, j, s, gap=3, width=3, min_n=1)
    assert two.tolist() == [[100, 102, 1000, 1002, 3, 3], [103, 105, 1003, 1005, 3, 3]]


def test_rejects_lists_not_in_diagonal_order():
    # the search's canonical (i, j) order is not (dt, idx1) order: such a list
    # (and one with a repeated entry) is refused instead of silently giving
    # split runs
    i = np.array([5, 5, 6], np.uint32)
    j = np.array([20, 30, 21], np.uint32)
    s = np.ones(3, np.uint16)
    with pytest.raises(ValueError):
        oracle.station_clusters(i, j, s, gap=3, width=2, min_n=1)
    with pytest.raises(ValueError):
        oracle.station_clusters(np.array([5, 5], np.uint32), np.array([20, 20], np.uint32),
                                np.ones(2, np.uint16), gap=3, width=2, min_n=1)
    o = np.lexsort((i, j - i))
    assert oracle.station_clusters(i[o], j[o], s[o], gap=3, width=2, min_n=1).tolist() == [[15, 15, 5, 6, 2, 2],
                                                                                          [25, 25, 5, 5, 1, 1]]


def test_empty_and_bad_arguments():
    e = np.zeros(0, np.uint32)
    assert oracle.station_clusters(e, e, np.zeros(0, np.uint16), gap=3, width=2, min_n=1).shape == (0, 6)
    with pytest.raises(ValueError):
        oracle.station_clusters(e, e, np.zeros(0, np.uint16), gap=0, width=2, min_n=1)
