"""CUDA path vs the CPU oracle, bit-exact (all integer work).

Every comparison is element by element on the same seeded synthetic inputs:
signatures [b, N], the canonical table listings (key, id) per table, the drop
mask, and the final (i, j, votes) list sorted by (i, j).
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


def _pad(K):
    return ((K + 7) // 8) * 8


def _searcher(p, **opts):
    from paper_1803_09835_gb300 import Searcher
    return Searcher(p, **opts)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _oracle_run(p, idx, K):
    keys = oracle.keys(p, np.ascontiguousarray(idx[:, :K]))
    d = oracle.drop(p, keys)
    return keys, d, oracle.search(p, keys, d)


def _assert_lists(got, want):
    gi, gj, gv = got
    wi, wj, wv = want
    assert len(gi) == len(wi), (len(gi), len(wi))
    assert np.array_equal(gi, wi) and np.array_equal(gj, wj) and np.array_equal(gv, wv)


SIG_CASES = [
    ("c0", dict(), 8192, None),                       # MinHash 16x4, D=2048, K=100, unaligned rows
    ("c0", dict(), 8192, 104),                         # padded rows -> 128-bit loads
    ("c1", dict(), 5000 + 13, 400),                    # Min-Max 100x4, ragged last tile
    ("c1", dict(r=3, b=30), 777, 408),                 # odd r: last function gives its min only
    ("c1", dict(K=40, b=12), 1000, 40),                # K^2 < D: direct-evaluation kernel
    ("c0", dict(kind=1, r=6, b=10), 33, 104),          # Min-Max on C0 shape, 2 tiles
]


@pytest.mark.parametrize("name,over,n,ld", SIG_CASES)
def test_signatures_bit_exact(name, over, n, ld):
    w = synth.scaled(name, n, **over)
    ld = ld or w.K
    idx = synth.generate(w, ld=ld)
    p = w.params()
    s = _searcher(p)
    sig = s.sig(torch.from_numpy(idx).cuda())
    want = oracle.keys(p, np.ascontiguousarray(idx[:, :w.K]))
    assert np.array_equal(_u32(sig), want)
    s.close()


def test_tables_and_filter_bit_exact():
    w = synth.scaled("c1", 60_000)
    idx = synth.generate(w, ld=400)
    p = w.params()
    s = _searcher(p)
    sig = s.sig(torch.from_numpy(idx).cuda())
    tb = s.build_tables(sig)
    keys = oracle.keys(p, idx)
    skey, sid, drop = _u32(tb.skey).reshape(p["b"], -1), _u32(tb.sid).reshape(p["b"], -1), tb.drop.cpu().numpy()
    for t in range(p["b"]):
        ok, oi = oracle.table(keys[t])
        assert np.array_equal(skey[t], ok) and np.array_equal(sid[t], oi), f"table {t}"
    want_drop = oracle.drop(p, keys)
    assert want_drop.sum() > 0
    assert np.array_equal(drop, want_drop)
    res = s.search(tb)
    _assert_lists(res.numpy(), oracle.search(p, keys, want_drop))
    tb.free()
    s.close()


DETECT_CASES = [
    ("c0", 8192, dict(), dict()),
    ("c0", 8192, dict(v=1, excl=0), dict(large_min=6)),
    ("c1", 60_000, dict(), dict()),
    ("c1", 60_000, dict(), dict(large_min=16)),               # dense groups on every large bucket
    ("c1", 60_000, dict(query_part=3), dict(map_load=0.8)),   # three row partitions of the pair buffer
    ("c1", 60_000, dict(query_part=7), dict(large_min=16)),   # seven partitions, dense groups everywhere
    ("c1", 40_000, dict(occ_num=0), dict(large_min=64)),      # no filter: the 60 s source stays
    ("c1", 20_000, dict(kind=0, r=2, b=40, v=3), dict()),     # MinHash on the C1 shape
    ("c1", 60_000, dict(), dict(vote_map=1)),                 # global vote map instead of per-row votes
    ("c1", 60_000, dict(query_part=4), dict(vote_map=1, large_min=10**9)),
    ("c1", 30_000, dict(occ_num=0), dict(large_min=10**9)),   # no dense groups: long rows per fingerprint
    ("c4", 50_000, dict(), dict()),                           # C4 shape: 30/60/90/3600 s sources, 200-repeat templates
    ("c4", 50_000, dict(query_part=5), dict(large_min=32)),   # C4 shape, five row partitions, dense groups
    # table groups (§6.4): tables sorted g at a time, votes over all of them
    ("c4", 50_000, dict(table_group=1), dict()),
    ("c4", 50_000, dict(table_group=3, query_part=5), dict()),
    ("c4", 50_000, dict(table_group=10), dict(large_min=32)),
    ("c4", 50_000, dict(table_group=10, query_part=5), dict()),
    ("c1", 20_000, dict(table_group=7), dict(single_pass=0)),  # 100 = 14 x 7 + 2: a short last group
    # imbalanced, co-occurring bits (§6.3): large background buckets
    ("c1", 30_000, dict(skew=0.6, corr=0.3), dict()),
    ("c1", 30_000, dict(skew=0.3, r=8, v=3), dict()),
    # a 4 s source without the filter: sparse buckets of up to 4,437 live
    # windows, more than the 4,096 a medium-bucket CTA holds by default
    ("c1", 28_000, dict(occ_num=0, b=20, v=2, periods=(4,)), dict(large_min=10**9)),
    ("c1", 28_000, dict(occ_num=0, b=20, v=2, periods=(4,)), dict(large_min=4500)),
]


@pytest.mark.parametrize("name,n,over,opts", DETECT_CASES)
def test_detections_bit_exact(name, n, over, opts):
    over = dict(over)
    qp = over.pop("query_part", 0)
    tg = over.pop("table_group", 0)
    w = synth.scaled(name, n, **over)
    idx = synth.generate(w, ld=_pad(w.K))
    p = dict(w.params(), query_part=qp, table_group=tg)
    s = _searcher(p, **opts)
    res = s.detect(torch.from_numpy(idx).cuda())
    got = res.numpy()
    _, _, want = _oracle_run(p, idx, w.K)
    assert len(want[0]) > 0
    _assert_lists(got, want)
    st = s.stats()
    assert st["n_detections"] == len(want[0])
    res.free()
    s.close()


def test_row_partitions_identical_and_forced_by_budget():
    # §6.4: the partitioned search yields the same list; a budget too small
    # for the whole pair buffer splits it without being asked
    from paper_1803_09835_gb300 import FastError, Searcher
    w = synth.scaled("c1", 40_000)
    idx = torch.from_numpy(synth.generate(w, ld=_pad(w.K))).cuda()
    p = w.params()
    s = _searcher(p)
    ref = s.detect(idx).numpy()
    st = s.stats()
    assert st["query_parts"] == 1
    peak, need = st["peak_bytes"], st["n_emissions"] * 4
    s.close()
    for qp in (2, 5):
        sq = _searcher(dict(p, query_part=qp))
        _assert_lists(sq.detect(idx).numpy(), ref)
        assert sq.stats()["query_parts"] == qp
        sq.close()
    # a budget-driven split needs the pair buffer to dominate memory: few
    # single-function MinHash tables collide often (~2.5 % per table here)
    from dataclasses import replace
    wb = replace(synth.scaled("c1", 20_000), n_templates=0, periods=(), kind=0, r=1, b=10, v=3, excl=0, occ_num=0)
    idxb = torch.from_numpy(synth.generate(wb, ld=_pad(wb.K))).cuda()
    pb = wb.params()
    # no dense groups: every pair goes through the pair buffer, counted then written
    s = _searcher(pb, large_min=10**9, single_pass=0)
    refb = s.detect(idxb).numpy()
    st = s.stats()
    peak, need = st["peak_bytes"], st["n_emissions"] * 4
    assert need > peak / 2 and len(refb[0]) > 0
    s.close()
    split = 0
    for frac in (0.3, 0.45, 0.6):
        sb = Searcher(pb, hbm_budget_bytes=int(peak - frac * need), large_min=10**9, single_pass=0)
        try:
            got = sb.detect(idxb).numpy()
        except FastError:
            sb.close()
            continue
        _assert_lists(got, refb)
        split += sb.stats()["query_parts"] >= 2
        sb.close()
    assert split >= 1


def test_dense_vote_fallback_and_budgets():
    # the branch taken when the cluster masks' scratch does not fit (every
    # dense group voted by direct comparison of the members' keys), forced by
    # the dense_masks option, gives the oracle's list; and for any HBM budget
    # from the unconstrained peak down the search either reports the budget
    # or gives the same list
    from paper_1803_09835_gb300 import FastError, Searcher, _lib
    w = synth.scaled("c1", 30_000)
    idx = synth.generate(w, ld=400)
    d = torch.from_numpy(idx).cuda()
    p = dict(w.params(), table_group=1)
    _, _, want = _oracle_run(p, idx, w.K)
    s = _searcher(p, large_min=16, dense_masks=0)
    r = s.detect(d)
    st = s.stats()
    assert st["n_groups"] > 0 and st["dense_fallback"] == 1
    _assert_lists(r.numpy(), want)
    r.free()
    s.close()
    s = _searcher(p, large_min=16)
    s.detect(d).free()
    st = s.stats()
    peak = st["peak_bytes"]
    assert st["n_groups"] > 0 and st["dense_fallback"] == 0
    s.close()
    ok = 0
    for k in range(24):
        sb = Searcher(p, hbm_budget_bytes=int(peak * (1 - 0.03 * k)), large_min=16)
        try:
            r = sb.detect(d)
        except FastError as e:
            assert e.status in (_lib.FAST_EBUDGET, _lib.FAST_ENOMEM)
            sb.close()
            continue
        _assert_lists(r.numpy(), want)
        r.free()
        ok += 1
        sb.close()
    assert ok > 1


@pytest.mark.parametrize("name,n,over", [("c1", 60_000, dict()), ("c0", 8192, dict(v=1, excl=0))])
def test_single_pass_and_overflow_identical(name, n, over):
    # pairs written once into fixed group regions (default), counted then
    # written (single_pass=0), and regions of 2 slots per group so that
    # almost every pair goes through the overflow list: one list
    w = synth.scaled(name, n, **over)
    idx = torch.from_numpy(synth.generate(w, ld=_pad(w.K))).cuda()
    p = w.params()
    lists = []
    for opts in (dict(), dict(single_pass=0), dict(group_slots=2), dict(group_slots=1, large_min=10**9)):
        s = _searcher(p, **opts)
        lists.append(s.detect(idx).numpy())
        s.close()
    assert len(lists[0][0]) > 0
    for got in lists[1:3]:
        _assert_lists(got, lists[0])
    _, _, want = _oracle_run(p, idx.cpu().numpy(), w.K)
    _assert_lists(lists[0], want)
    _assert_lists(lists[3], want)


def test_dense_and_sparse_paths_agree():
    w = synth.scaled("c1", 50_000, occ_num=0)
    idx = torch.from_numpy(synth.generate(w, ld=400)).cuda()
    out = []
    for lm, vm in ((0, 0), (10, 0), (100, 0), (10**9, 0), (0, 1), (10**9, 1)):
        s = _searcher(w.params(), large_min=lm, vote_map=vm)
        r = s.detect(idx)
        out.append((r.numpy(), s.stats()))
        r.free()
        s.close()
    for o, st in out[1:]:
        _assert_lists(o, out[0][0])
    assert out[1][1]["n_groups"] > 0 and out[3][1]["n_groups"] == 0 and out[5][1]["n_groups"] == 0


def test_host_entry_point_matches_device():
    w = synth.scaled("c1", 30_000)
    idx = synth.generate(w, ld=400)
    s = _searcher(w.params())
    r = s.detect(torch.from_numpy(idx).cuda())
    dev = r.numpy()
    M, i, j, v = s.detect_host(idx, cap=len(dev[0]) + 5)
    assert M == len(dev[0])
    _assert_lists((i, j, v), dev)
    M2, i2, _, _ = s.detect_host(idx, cap=7)  # truncated copy keeps the first cap in order
    assert M2 == M and np.array_equal(i2, dev[0][:7])
    r.free()
    s.close()


def _filler(w, ld):
    def fill(r0, n, rows):
        synth.generate(w, ld=ld, out=rows, rows=(r0, r0 + n))
    return fill


@pytest.mark.parametrize("n,tg,qp,chunk", [(50_000, 10, 0, 7001), (300_000, 10, 5, 65_536), (40_000, 0, 0, 40_000)])
def test_chunked_host_input_c4_shape(n, tg, qp, chunk):
    # §6.4: a station too long to hold at once, fed in chunks, with its tables
    # sorted 10 at a time and its pair buffer split into query partitions
    w = synth.scaled("c4", n)
    p = dict(w.params(), table_group=tg, query_part=qp)
    s = _searcher(p)
    r = s.detect_chunked(w.N, 400, _filler(w, 400), chunk_rows=chunk)
    got = r.numpy()
    r.free()
    idx = synth.generate(w, ld=400)
    _, _, want = _oracle_run(p, idx, w.K)
    assert len(want[0]) > 0
    _assert_lists(got, want)
    s.close()


def test_chunked_signatures_and_fill_failure():
    from paper_1803_09835_gb300 import FastError
    w = synth.scaled("c1", 20_000)
    idx = synth.generate(w, ld=408)
    p = w.params()
    s = _searcher(p)
    sig = torch.empty((p["b"], w.N), dtype=torch.int32, device="cuda")
    for r0, r1 in ((0, 5003), (5003, 5003), (5003, 17_777), (17_777, 20_000)):
        s.sig_rows(torch.from_numpy(idx[r0:r1]).cuda(), sig, r0)
    assert np.array_equal(_u32(sig), oracle.keys(p, np.ascontiguousarray(idx[:, :w.K])))
    with pytest.raises(FastError):
        s.sig_rows(torch.from_numpy(idx[:10]).cuda(), sig, w.N - 5)  # past the end

    def bad(r0, n, rows):
        if r0 > 0:
            raise RuntimeError("fingerprint source gone")
        rows[:] = idx[r0:r0 + n]
    with pytest.raises(RuntimeError):
        s.detect_chunked(w.N, 408, bad, chunk_rows=6000)
    good = s.detect_chunked(w.N, 408, lambda r0, n, rows: rows.__setitem__(slice(None), idx[r0:r0 + n]),
                            chunk_rows=6000)
    _, _, want = _oracle_run(p, idx, w.K)
    _assert_lists(good.numpy(), want)
    good.free()
    s.close()


# ------------------------------------------------------------ edge cases

def _params(**kw):
    p = dict(D=2048, K=100, b=16, r=4, kind=0, seed=7, v=2, excl=0, occ_num=0, occ_den=1000)
    p.update(kw)
    return p


def test_empty_and_tiny_inputs():
    p = _params()
    s = _searcher(p)
    for n in (0, 1):
        r = s.detect(torch.zeros((n, 104), dtype=torch.int16, device="cuda").view(torch.uint16)
                     if n == 0 else torch.from_numpy(np.arange(104, dtype=np.uint16)[None]).cuda())
        assert r.M == 0
        r.free()
    two = np.stack([np.arange(100, dtype=np.uint16)] * 2)
    r = s.detect(torch.from_numpy(two).cuda())
    i, j, v = r.numpy()
    assert list(zip(i, j, v)) == [(0, 1, 16)]
    r.free()
    s.close()


@pytest.mark.parametrize("lm", [0, 4, 10**9])
def test_identical_fingerprints_one_giant_bucket(lm):
    p = _params(excl=3, v=16)
    n = 700
    idx = np.tile(np.arange(0, 2000, 20, dtype=np.uint16), (n, 1))
    s = _searcher(p, large_min=lm)
    r = s.detect(torch.from_numpy(idx).cuda())
    i, j, v = r.numpy()
    keys = oracle.keys(p, idx)
    want = oracle.search(p, keys, None)
    _assert_lists((i, j, v), want)
    assert len(i) == sum(n - 1 - a - 3 for a in range(n - 4))
    r.free()
    s.close()


def test_filter_that_drops_everything():
    w = synth.scaled("c1", 5000, occ_num=1, occ_den=10 * 5000)
    idx = synth.generate(w, ld=400)
    s = _searcher(w.params())
    r = s.detect(torch.from_numpy(idx).cuda())
    assert r.M == 0 and s.stats()["n_dropped"] == 5000
    r.free()
    s.close()


def test_bad_index_is_reported_and_context_survives():
    from paper_1803_09835_gb300 import FastError, _lib
    p = _params()
    s = _searcher(p)
    idx = np.tile(np.arange(100, dtype=np.uint16), (64, 1))
    idx[5, 7] = 2048  # == D
    with pytest.raises(FastError) as e:
        s.detect(torch.from_numpy(idx).cuda())
    assert e.value.status == _lib.FAST_EINVAL
    idx[5, 7] = 2047
    r = s.detect(torch.from_numpy(idx).cuda())
    assert r.M > 0
    r.free()
    s.close()


@pytest.mark.parametrize("bad", [dict(b=0), dict(b=256), dict(v=17), dict(r=0), dict(K=3000), dict(kind=2),
                                 dict(occ_num=1, occ_den=0), dict(D=70000), dict(table_group=17)])
def test_invalid_parameters(bad):
    from paper_1803_09835_gb300 import FastError
    with pytest.raises(FastError):
        _searcher(_params(**bad))


def test_hbm_budget_is_enforced():
    from paper_1803_09835_gb300 import FastError, _lib
    from paper_1803_09835_gb300 import Searcher
    w = synth.scaled("c1", 20_000)
    idx = torch.from_numpy(synth.generate(w, ld=400)).cuda()
    s = Searcher(w.params(), hbm_budget_bytes=1 << 20)
    with pytest.raises(FastError) as e:
        s.detect(idx)
    assert e.value.status == _lib.FAST_EBUDGET
    s.close()


# ------------------------------------------------------ full-size workload

@pytest.mark.slow
def test_c1_full_size_sampled_rows():
    """The 3-month, 7.776M-window workload in the benchmark's configuration;
    the oracle recomputes every key and checks sampled rows and entries."""
    w = synth.workload("c1")
    idx = synth.generate(w, ld=400)
    p = w.params()
    s = _searcher(p)
    r = s.detect(torch.from_numpy(idx).cuda())
    gi, gj, gv = r.numpy()
    st = s.stats()
    r.free()
    s.close()
    torch.cuda.empty_cache()
    # structural properties of the whole list
    assert len(gi) > 10**8
    assert np.all(gi < gj) and np.all(gj.astype(np.int64) - gi > p["excl"]) and np.all(gv >= p["v"])
    key = (gi.astype(np.uint64) << np.uint64(32)) | gj
    assert np.all(key[1:] > key[:-1])
    keys = oracle.keys(p, idx)
    drop = oracle.drop(p, keys)
    assert st["n_dropped"] == int(drop.sum())
    assert not drop[gi].any() and not drop[gj].any()
    rng = np.random.default_rng(0)
    # sampled rows: some with detections (noise / template copies), some random
    rows = np.concatenate([rng.choice(np.unique(gi[::9973]), 12, replace=False), rng.integers(0, w.N, 8)])
    starts = np.searchsorted(gi, rows)
    ends = np.searchsorted(gi, rows, side="right")
    for row, a, b in zip(rows, starts, ends):
        wj, wv = oracle.search_row(p, keys, drop, int(row))
        assert np.array_equal(gj[a:b], wj) and np.array_equal(gv[a:b], wv), f"row {row}"
    # sampled entries: votes from the definition
    for x in rng.integers(0, len(gi), 3000):
        assert oracle.pair_votes(p, keys, int(gi[x]), int(gj[x])) == gv[x]


@pytest.mark.slow
def test_c4_full_size_chunked_table_groups():
    """The 5-year, 157,680,000-window station: input generated and fed in
    chunks, tables sorted 10 at a time (the configuration's 10 groups of 10),
    the pair buffer in as many query partitions as the device needs.  The
    oracle cannot hold this station's keys, so the list is checked by its
    invariants, by exact votes of sampled entries (keys of the two windows
    from the oracle), and by recall on sampled candidate pairs (copies of one
    template or of the hourly / daily sources): a pair of live windows is in
    the list exactly when the oracle counts >= v shared tables."""
    w = synth.workload("c4")
    p = dict(w.params(), table_group=10)
    s = _searcher(p)
    r = s.detect_chunked(w.N, 400, _filler(w, 400), chunk_rows=1 << 22)
    gi, gj, gv = r.numpy()
    st = s.stats()
    r.free()
    s.close()
    torch.cuda.empty_cache()
    assert len(gi) > 10**8 and st["n_dropped"] > 0
    assert np.all(gi < gj) and np.all(gj.astype(np.int64) - gi > p["excl"])
    assert np.all(gv >= p["v"]) and np.all(gv <= p["b"])
    key = (gi.astype(np.uint64) << np.uint64(32)) | gj
    assert np.all(key[1:] > key[:-1])
    del key
    rng = np.random.default_rng(4)

    def keys_of(ids):
        return oracle.keys(p, synth.generate_ids(w, np.asarray(ids, np.uint64), ld=400))

    # exact votes of sampled entries
    xs = rng.integers(0, len(gi), 2000)
    ki, kj = keys_of(gi[xs]), keys_of(gj[xs])
    assert np.array_equal((ki == kj).sum(axis=0), gv[xs])
    # recall on candidate pairs among windows of one template or source that
    # the filter cannot touch (sources repeating more often than every 200 s
    # are the only ones whose buckets can exceed 0.5 % of the station)
    own = synth.owners(w)
    groups = {}
    for code in (synth.OWNER_PERIODIC + 3, synth.OWNER_PERIODIC + 4):  # 3600 s and 86400 s sources
        groups[code] = np.nonzero(own == code)[0]
    tpl = own[own >= synth.OWNER_TEMPLATE]
    for t in rng.choice(np.unique(tpl), 40, replace=False):
        groups[int(t)] = np.nonzero(own == t)[0]
    cand = []
    for ids in groups.values():
        if len(ids) < 2:
            continue
        for _ in range(25):
            a, b = np.sort(rng.choice(ids, 2, replace=False))
            if b - a > p["excl"]:
                cand.append((a, b))
    cand = np.array(cand, np.int64)
    ka, kb = keys_of(cand[:, 0]), keys_of(cand[:, 1])
    votes = (ka == kb).sum(axis=0)
    key = gi.astype(np.int64) * (1 << 32) + gj
    want = cand[:, 0] * (1 << 32) + cand[:, 1]
    pos = np.minimum(np.searchsorted(key, want), len(key) - 1)
    found = key[pos] == want
    assert np.array_equal(found, votes >= p["v"]), (found.sum(), (votes >= p["v"]).sum())
    assert found.sum() > 0
