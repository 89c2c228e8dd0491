"""The shared synthetic input generator (CPU only)."""
import numpy as np

import synth


def test_rows_are_sorted_k_subsets_and_reproducible():
    w = synth.scaled("c1", 20_000)
    a = synth.generate(w, threads=3)
    b = synth.generate(w, threads=5)
    assert np.array_equal(a, b)
    assert a.shape == (20_000, 400)
    assert np.all(np.diff(a.astype(np.int32), axis=1) > 0)
    assert a.max() < w.D


def test_padding_and_owner_structure():
    w = synth.scaled("c1", 30_000)
    idx, own = synth.generate(w, ld=408, owner=True)
    assert np.all(idx[:, 400:] == 0xFFFF)
    per = own[(own >= synth.OWNER_PERIODIC) & (own < synth.OWNER_TEMPLATE)] - synth.OWNER_PERIODIC
    assert set(np.unique(per).tolist()) == {0, 1, 2}
    # periodic copies recur every P windows unless a template overwrote them
    for p, P in enumerate(w.periods):
        pos = np.nonzero(own == synth.OWNER_PERIODIC + p)[0]
        assert np.all(np.diff(pos) % P == 0)
        assert len(pos) >= 0.9 * (w.N // P)


def test_noisy_copies_keep_k_and_overlap():
    w = synth.scaled("c1", 30_000)
    idx, own = synth.generate(w, owner=True)
    pos = np.nonzero(own == synth.OWNER_PERIODIC + 1)[0][:20]  # the 300 s source, 5 % re-draw
    for x in pos[1:]:
        inter = len(np.intersect1d(idx[pos[0]], idx[x]))
        assert inter >= 400 - 2 * 20  # each copy re-draws 20 of 400 bits


def test_shared_templates_across_stations():
    a, oa = synth.generate(synth.scaled("c2", 40_000, station=0), owner=True)
    b, ob = synth.generate(synth.scaled("c2", 40_000, station=3), owner=True)
    ta = set((oa[oa >= synth.OWNER_TEMPLATE] - synth.OWNER_TEMPLATE).tolist())
    tb = set((ob[ob >= synth.OWNER_TEMPLATE] - synth.OWNER_TEMPLATE).tolist())
    assert len(ta & tb) > 0


def test_request_schedule():
    t, st, size = synth.requests(5000, 2000.0)
    assert np.all(np.diff(t) >= 0) and abs(5000 / t[-1] - 2000) < 200
    assert size.min() >= 60 and size.max() <= 3600 and st.max() < 12


def test_row_ranges_equal_the_whole_station():
    # a large station is drawn chunk by chunk: any row range must be exactly
    # those rows of the whole station (periodic phases, template placements)
    w = synth.scaled("c4", 50_000)
    full, own = synth.generate(w, ld=408, owner=True)
    for r0, r1 in ((0, 50_000), (0, 1), (17, 4113), (29_999, 50_000), (12_345, 12_345)):
        part, po = synth.generate(w, ld=408, owner=True, rows=(r0, r1))
        assert part.shape == (r1 - r0, 408)
        assert np.array_equal(part, full[r0:r1]) and np.array_equal(po, own[r0:r1])
    import pytest
    with pytest.raises(ValueError):
        synth.generate(w, rows=(10, 50_001))


def _bit_stats(a, D=8192, top=300):
    f = np.bincount(a.ravel(), minlength=D) / len(a)
    idx = np.argsort(f)[::-1][:top]
    m = np.zeros((len(a), D), bool)
    m[np.arange(len(a))[:, None], a] = True
    x = m[:, idx].astype(np.float64)
    p = x.mean(0)
    lift = (x.T @ x / len(a)) / np.outer(p, p)
    np.fill_diagonal(lift, 0)
    return f, lift


def test_skewed_and_correlated_bits():
    # §6.3: some fingerprint elements are non-zero far more often than
    # others, and some co-occur; the generator's skew and corr draw that
    from dataclasses import replace
    w = replace(synth.scaled("c1", 20_000), n_templates=0, periods=())
    uni = synth.generate(w)
    assert np.array_equal(uni, synth.generate(replace(w, skew=0.0, corr=0.0)))
    f0, l0 = _bit_stats(uni)
    assert f0.max() < 0.1 and l0.max() < 2.0
    sk = synth.generate(replace(w, skew=0.6))
    assert np.all(np.diff(sk.astype(np.int32), axis=1) > 0) and sk.max() < w.D
    f1, l1 = _bit_stats(sk)
    top1 = np.sort(f1)[::-1][:w.D // 100].sum() / f1.sum()
    assert f1.max() > 0.5 and top1 > 5 * 0.01 * 1.5  # the top 1 % of bits hold several times their share
    assert l1.max() < 1.5                            # imbalance alone adds no co-occurrence
    co = synth.generate(replace(w, skew=0.6, corr=0.5))
    _, l2 = _bit_stats(co)
    assert l2.max() > 3.0                            # partners co-occur
    # noisy copies keep exactly K bits under the skew too
    ws = replace(synth.scaled("c1", 20_000), skew=0.6, corr=0.3)
    a, own = synth.generate(ws, owner=True)
    assert np.all(np.diff(a.astype(np.int32), axis=1) > 0)
    assert (own >= synth.OWNER_TEMPLATE).sum() > 0


def test_owners_only_and_listed_windows():
    # the source codes alone, and arbitrary lists of windows, equal the whole
    # station's (the full-size tests draw sampled windows this way)
    for name, n in (("c4", 60_000), ("c2", 50_000)):
        w = synth.scaled(name, n, station=3) if name == "c2" else synth.scaled(name, n)
        full, own = synth.generate(w, ld=400, owner=True)
        assert np.array_equal(synth.owners(w), own)
        assert np.array_equal(synth.owners(w, rows=(1234, 40_000)), own[1234:40_000])
        rng = np.random.default_rng(3)
        ids = np.concatenate([rng.integers(0, n, 500), np.nonzero(own >= synth.OWNER_TEMPLATE)[0][:100],
                              np.nonzero((own >= synth.OWNER_PERIODIC) & (own < synth.OWNER_TEMPLATE))[0][:50],
                              [0, n - 1, 7, 7]])
        assert np.array_equal(synth.generate_ids(w, ids, ld=400), full[ids])
    from dataclasses import replace
    ws = replace(synth.scaled("c1", 20_000), skew=0.6, corr=0.3)
    full = synth.generate(ws)
    ids = np.array([19_999, 5, 5, 12_345])
    assert np.array_equal(synth.generate_ids(ws, ids), full[ids])
