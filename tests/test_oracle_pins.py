"""Pins of the CPU oracle to facts outside itself (CPU only).

Nothing here asserts the oracle against a retyped copy of its own formulas.
The pins are: published SplitMix64 outputs, arithmetic properties of a
multiply-add-shift map, algebraic invariants of min/max over sets, the
MinHash / Min-Max collision laws and the detection S-curve of §6.3 (closed
forms), and brute force over all pairs on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
M32 = (1 << 32) - 1


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        s, n, v = line.split()
        rows.append((int(s), int(n), int(v, 0)))
    return rows


def P(**kw):
    p = dict(D=2048, K=100, b=16, r=4, kind=0, seed=0x1803098350, v=2, excl=5, occ_num=0, occ_den=1000)
    p.update(kw)
    return p


# ---------------------------------------------------------------- hashing

def test_splitmix64_published_outputs():
    for seed, n, v in _golden():
        assert oracle.sm64(seed, n) == v


def test_hash_parameters_come_from_the_published_stream():
    g = {(s, n): v for s, n, v in _golden()}
    a, b = oracle.hash_params(P(seed=1234567, b=1, r=2, kind=1))  # F = 1
    assert int(a[0]) == g[(1234567, 0)] | 1 and int(b[0]) == g[(1234567, 1)]
    a, b = oracle.hash_params(P(seed=1234567, b=2, r=1, kind=0))  # F = 2
    assert int(a[1]) == g[(1234567, 2)] | 1 and int(b[1]) == g[(1234567, 3)]
    assert all(int(x) & 1 for x in a)


@pytest.mark.parametrize("kind,b,r", [(0, 16, 4), (1, 100, 4), (1, 3, 3)])
def test_number_of_functions(kind, b, r):
    # MinHash needs r functions per table; Min-Max keeps min and max and needs
    # ceil(r/2) (§6.2 "halves the number of hash functions"; Algorithm 1).
    F = oracle.nfuncs(P(kind=kind, b=b, r=r))
    assert F == (b * r if kind == 0 else b * ((r + 1) // 2))


def test_h_is_the_top_half_of_an_affine_progression():
    # For y(x) = a*x + b mod 2^64, y(x+1) - y(x) = a, so the top 32 bits step by
    # a>>32 or a>>32 + 1 (carry), and h(0) = b>>32.  A wrong shift, a dropped
    # +b, swapped a/b or a 32-bit product all break this.
    D = 8192
    p = P(D=D, K=1, b=4, r=4, kind=0)
    a, b = oracle.hash_params(p)
    xs = np.arange(D, dtype=np.uint16)[:, None]
    mn, _ = oracle.values(p, xs)  # K=1: mn[x, f] = h_f(x)
    for f in range(len(a)):
        h = mn[:, f].astype(np.int64)
        assert h[0] == int(b[f]) >> 32
        step = np.diff(h) % (1 << 32)
        ahi = int(a[f]) >> 32
        assert set(np.unique(step).tolist()) <= {ahi, (ahi + 1) & M32}
        # the number of carries over D steps is fixed by the low halves
        lo_a, lo_b = int(a[f]) & M32, int(b[f]) & M32
        carries = (lo_a * (D - 1) + lo_b) >> 32
        assert int(np.sum(step == ((ahi + 1) & M32))) == carries


# ---------------------------------------------------------- min / max of sets

def _rand_sets(rng, n, D, K):
    return np.stack([np.sort(rng.choice(D, K, replace=False)) for _ in range(n)]).astype(np.uint16)


def test_minmax_invariants():
    rng = np.random.default_rng(3)
    D, K = 2048, 64
    p = P(D=D, K=K, b=8, r=4, kind=1)
    A = _rand_sets(rng, 20, D, K)
    mn, mx = oracle.values(p, A)
    assert np.all(mn <= mx)
    # permutation invariance: the row order of the set does not matter
    Ash = np.stack([rng.permutation(r) for r in A])
    mn2, mx2 = oracle.values(p, Ash)
    assert np.array_equal(mn, mn2) and np.array_equal(mx, mx2)
    # K = 1: min = max = h(x)
    p1 = dict(p, K=1)
    m1, x1 = oracle.values(p1, A[:, :1].copy())
    assert np.array_equal(m1, x1)
    # union property and subset monotonicity
    B = _rand_sets(rng, 20, D, K)
    for r in range(20):
        U = np.union1d(A[r], B[r]).astype(np.uint16)
        mu, xu = oracle.values(dict(p, K=len(U)), U[None, :])
        assert np.array_equal(mu[0], np.minimum(mn[r], oracle.values(p, B[r:r + 1])[0][0]))
        assert np.array_equal(xu[0], np.maximum(mx[r], oracle.values(p, B[r:r + 1])[1][0]))
        S = A[r, :K // 2].copy()
        ms, xs = oracle.values(dict(p, K=len(S)), S[None, :])
        assert np.all(mn[r] <= ms[0]) and np.all(mx[r] >= xs[0])


def _pair_with_overlap(rng, D, K, c):
    perm = rng.permutation(D)
    A = np.sort(perm[:K])
    B = np.sort(np.concatenate([perm[:c], perm[K:2 * K - c]]))
    return A.astype(np.uint16), B.astype(np.uint16)


@pytest.mark.parametrize("c", [40, 200, 320, 380])
def test_per_function_collision_laws(c):
    # MinHash: P[min_A = min_B] = J = c/u (§6.1, Broder).  Min-Max: min and max
    # of A u B under a random order form a uniform ordered pair of distinct
    # elements, so P[min and max agree] = c(c-1) / (u(u-1)) (§6.2).
    rng = np.random.default_rng(c)
    D, K = 8192, 400
    u = 2 * K - c
    n = hit_min = hit_mm = 0
    for trial in range(12):
        p = P(D=D, K=K, b=2000, r=2, kind=1, seed=1000 + trial)
        A, B = _pair_with_overlap(rng, D, K, c)
        (ma, xa), (mb, xb) = oracle.values(p, A[None]), oracle.values(p, B[None])
        hit_min += int(np.sum(ma == mb))
        hit_mm += int(np.sum((ma == mb) & (xa == xb)))
        n += ma.size
    for got, want in ((hit_min / n, c / u), (hit_mm / n, c * (c - 1) / (u * (u - 1)))):
        assert abs(got - want) <= 4 * math.sqrt(want * (1 - want) / n) + 1e-12, (got, want)


def test_keys_collide_exactly_when_bands_agree():
    # key_t(i) = key_t(j) iff the table's r band values agree (up to 2^-32):
    # pins which functions feed which table and the order min, max, min, max.
    rng = np.random.default_rng(11)
    for kind, b, r in ((0, 16, 4), (1, 25, 4), (1, 10, 3)):
        D, K = 2048, 100
        p = P(D=D, K=K, b=b, r=r, kind=kind)
        base = np.sort(rng.choice(D, K, replace=False))
        rows = [base]
        for m in (1, 2, 3, 5, 8, 13):  # near-duplicates share many band values
            keep = rng.choice(K, K - m, replace=False)
            rest = np.setdiff1d(np.arange(D), base[keep])
            rows.append(np.sort(np.concatenate([base[keep], rng.choice(rest, m, replace=False)])))
        X = np.stack(rows).astype(np.uint16)
        mn, mx = oracle.values(p, X)
        keys = oracle.keys(p, X)
        q = (r + 1) // 2
        for t in range(b):
            if kind == 0:
                band = mn[:, t * r:(t + 1) * r]
            else:
                cols = []
                for cidx in range(r):
                    f = t * q + cidx // 2
                    cols.append(mn[:, f] if cidx % 2 == 0 else mx[:, f])
                band = np.stack(cols, 1)
            for i in range(len(X)):
                for j in range(i + 1, len(X)):
                    assert (keys[t, i] == keys[t, j]) == bool(np.all(band[i] == band[j]))


def _scurve(s_r, t, m):
    # §6.3: P[s] = 1 - sum_{i<m} C(t,i) (1 - s^k)^(t-i) (s^k)^i, with s^k the
    # per-table collision probability.
    return 1 - sum(math.comb(t, i) * (1 - s_r) ** (t - i) * s_r ** i for i in range(m))


def test_vote_distribution_follows_the_scurve():
    # Tables use disjoint functions, so the number of colliding tables of a
    # pair is Binomial(b, p_table) and P[votes >= v] is the S-curve of §6.3.
    rng = np.random.default_rng(5)
    D, K, b, r, v = 8192, 400, 100, 4, 4
    for c in (280, 330):
        u = 2 * K - c
        p_tab = (c * (c - 1) / (u * (u - 1))) ** 2
        votes = []
        for trial in range(60):
            p = P(D=D, K=K, b=b, r=r, kind=1, seed=77 + trial)
            A, B = _pair_with_overlap(rng, D, K, c)
            k = oracle.keys(p, np.stack([A, B]))
            votes.append(int(np.sum(k[:, 0] == k[:, 1])))
        votes = np.array(votes)
        n = len(votes) * b
        mean_p = votes.sum() / n
        assert abs(mean_p - p_tab) <= 4 * math.sqrt(p_tab * (1 - p_tab) / n)
        want = _scurve(p_tab, b, v)
        got = float(np.mean(votes >= v))
        assert abs(got - want) <= 4 * math.sqrt(want * (1 - want) / len(votes)) + 0.02


# ------------------------------------------------------------ tables, filter

def test_table_is_sorted_grouping():
    rng = np.random.default_rng(2)
    k = rng.integers(0, 50, 3000).astype(np.uint32)
    sk, si = oracle.table(k)
    assert np.array_equal(sk, k[si])
    order = np.lexsort((np.arange(3000), k))
    assert np.array_equal(si, order.astype(np.uint32))


def _near_dup_workload(N=400, seed=9):
    w = synth.Workload("tiny", N, 1024, 40, 12, 2, 1, 2, 2, 0, 1000, seed, periods=(7, 23),
                       per_redraw=0.05, n_templates=6, rep_lo=3, rep_hi=9, tpl_redraw=0.1, tpl_seed=seed)
    return w, synth.generate(w)


@pytest.mark.parametrize("num,den", [(5, 100), (1, 40), (3, 1000)])
def test_occurrence_filter_brute_force(num, den):
    w, idx = _near_dup_workload()
    p = dict(w.params(), occ_num=num, occ_den=den)
    keys = oracle.keys(p, idx)
    N, b = idx.shape[0], p["b"]
    cnt = np.zeros(N, np.int64)
    for t in range(b):
        for i in range(N):
            size = int(np.sum(keys[t] == keys[t, i]))
            cnt[i] += den * size > num * N
    d, c = oracle.drop(p, keys, heavy_cnt=True)
    assert np.array_equal(c, cnt)
    assert np.array_equal(d, (2 * cnt > b).astype(np.uint8))
    assert d.sum() > 0  # the periodic sources trip the filter


def test_occurrence_filter_limits():
    w, idx = _near_dup_workload()
    p = w.params()
    keys = oracle.keys(p, idx)
    assert oracle.drop(dict(p, occ_num=0), keys).sum() == 0  # off
    assert oracle.drop(dict(p, occ_num=1, occ_den=1), keys).sum() == 0  # size > N impossible
    allheavy = dict(p, occ_num=1, occ_den=10 * idx.shape[0])  # every bucket heavy
    d = oracle.drop(allheavy, keys)
    assert d.sum() == idx.shape[0]
    i, j, v = oracle.search(allheavy, keys, d)
    assert len(i) == 0


# ------------------------------------------------------------------- search

@pytest.mark.parametrize("kind,r,v,excl,occ", [(0, 4, 2, 5, 0), (1, 4, 2, 0, 0), (1, 2, 1, 3, 5),
                                               (0, 1, 3, 0, 2), (1, 3, 2, 10, 0)])
def test_bucket_search_equals_brute_force(kind, r, v, excl, occ):
    w, idx = _near_dup_workload(N=500, seed=21 + r)
    p = dict(w.params(), kind=kind, r=r, v=v, excl=excl, occ_num=occ, occ_den=100)
    keys = oracle.keys(p, idx)
    d = oracle.drop(p, keys)
    got = oracle.search(p, keys, d)
    want = oracle.search(p, keys, d, brute=True)
    for g, x in zip(got, want):
        assert np.array_equal(g, x)
    i, j, vv = got
    assert len(i) > 0
    assert np.all(i < j) and np.all(j.astype(np.int64) - i > excl) and np.all(vv >= v)
    assert not np.any(d[i]) and not np.any(d[j])
    key = i.astype(np.uint64) << np.uint64(32) | j
    assert np.all(np.diff(key.astype(np.int64)) > 0)


def test_c0_bucket_search_equals_brute_force():
    w = synth.workload("c0")
    idx = synth.generate(w)
    p = w.params()
    keys = oracle.keys(p, idx)
    got = oracle.search(p, keys, None)
    want = oracle.search(p, keys, None, brute=True)
    for g, x in zip(got, want):
        assert np.array_equal(g, x)


def test_rows_match_the_full_list():
    w, idx = _near_dup_workload(N=600, seed=4)
    p = dict(w.params(), occ_num=5, occ_den=100)
    keys = oracle.keys(p, idx)
    d = oracle.drop(p, keys)
    i, j, v = oracle.search(p, keys, d)
    for row in np.unique(i)[:40]:
        jj, vv = oracle.search_row(p, keys, d, int(row))
        assert np.array_equal(jj, j[i == row]) and np.array_equal(vv, v[i == row])
        for a, b_ in zip(jj[:5], vv[:5]):
            assert oracle.pair_votes(p, keys, int(row), int(a)) == b_


def test_template_pairs_are_detected_at_the_scurve_rate():
    # End-to-end sanity on C0: copies of one template are detected with the
    # probability the S-curve gives for their actual overlap.
    w = synth.workload("c0")
    idx, owner = synth.generate(w, owner=True)
    p = w.params()
    keys = oracle.keys(p, idx)
    i, j, v = oracle.search(p, keys, None)
    found = set(zip(i.tolist(), j.tolist()))
    tpl = np.nonzero(owner >= synth.OWNER_TEMPLATE)[0]
    exp = var = 0.0
    hits = 0
    for a in range(len(tpl)):
        for c_ in range(a + 1, len(tpl)):
            x, y = int(tpl[a]), int(tpl[c_])
            if owner[x] != owner[y] or y - x <= p["excl"]:
                continue
            inter = len(np.intersect1d(idx[x], idx[y]))
            J = inter / (2 * p["K"] - inter)
            q = _scurve(J ** p["r"], p["b"], p["v"])
            exp += q
            var += q * (1 - q)
            hits += (x, y) in found
    assert exp > 500
    assert abs(hits - exp) <= 4 * math.sqrt(var) + 0.02 * exp
