/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the LSH similarity
 * search over binary waveform fingerprints (Rong et al., "Locality-Sensitive
 * Hashing for Earthquake Detection", §6).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path: every
 * formula below is written out here a second time, on purpose.
 *
 * What it computes, step by step, in the paper's order:
 *   1. hash mappings  h_f(x), f = 0..F-1       (§6.1 "Hash signature generation";
 *                                                Algorithm 1, single_hash)
 *   2. per-function min (MinHash) or min and max (Min-Max hash) of h_f over the
 *      fingerprint's non-zero positions          (§6.1; §6.2 Min-Max; Algorithm 1)
 *   3. one bucket key per (fingerprint, table) by combining the table's r values
 *                                                (Algorithm 1, hash_combine)
 *   4. hash tables: fingerprints grouped by equal key, per table
 *                                                (§6.1 "Hash table construction")
 *   5. occurrence filter                         (§6.5 "Removing correlated noise")
 *   6. votes(i,j) = number of tables in which i and j share a bucket, kept when
 *      votes >= v and j - i > E                  (§6.1 "Search"; §6.3 detection
 *                                                equation; §7.2 output triplets)
 *   7. (streaming replay of one request, section 7 below)
 *   8. channel level: the channels' lists summed by sort-merge-reduce and
 *      thresholded again                         (§7.1 "Channel Level"; §7.2,
 *                                                the sort-merge-reduce procedure)
 *   9. station level: thin diagonal clusters with summary statistics
 *                                                (§7.1 "Station Level"; §7.2)
 *
 * The paper leaves the hash family, hash_combine and the exact filter rule
 * open; the readings fixed here are:
 *   - SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) draws the hash parameters:
 *     sm64(seed, n) = mix64(seed + (n+1)*GAMMA), mix64 the SplitMix64 finaliser.
 *   - a_f = sm64(seed, 2f) | 1, b_f = sm64(seed, 2f+1),
 *     h_f(x) = high 32 bits of (a_f * x + b_f) mod 2^64   (multiply-add-shift).
 *   - MinHash: F = b*r functions; table t takes the minima of f = t*r .. t*r+r-1.
 *     Min-Max: F = b*ceil(r/2) functions; table t takes, for f = t*q .. t*q+q-1
 *     (q = ceil(r/2)), the sequence min_f, max_f, ... truncated to r values.
 *   - key_t = high 32 bits of z, where z starts at sm64(seed, 2F + t) and is
 *     folded with every band value w in order as z = mix64(z ^ w).
 *   - occurrence filter (static form): size_t(k) counts all N fingerprints;
 *     a bucket is heavy iff occ_den*size > occ_num*N; a fingerprint is dropped
 *     iff it lies in a heavy bucket in strictly more than b/2 tables.
 *     occ_num == 0 switches the filter off.
 *   - a pair (i, j), i < j, is reported iff neither is dropped, j - i > E and
 *     votes >= v.  Output is sorted by (i, j).
 *
 * Parity unpinned: the absolute hash and key VALUES follow only from the
 * readings above (the paper prints no worked example); tests pin them to the
 * published SplitMix64 outputs, to arithmetic-progression properties of the
 * multiply-add-shift, and to the collision laws of MinHash / Min-Max.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

typedef struct {
    uint32_t D, K, b, r, kind; /* kind: 0 = MinHash, 1 = Min-Max hash */
    uint64_t seed;
    uint32_t v, excl, occ_num, occ_den;
} orc_params;

/* ------------------------------------------------------------------ */
/* 1. random draws and the hash mappings                               */
/* ------------------------------------------------------------------ */

/* SplitMix64 finaliser (Steele, Lea & Flood 2014, the "mix64" variant). */
uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n-th SplitMix64 output of the generator seeded with `seed`. */
uint64_t orc_sm64(uint64_t seed, uint64_t n)
{
    return orc_mix64(seed + (n + 1) * ORC_GAMMA);
}

/* Number of hash functions F for the table layout of §6.1 / §6.2. */
uint32_t orc_nfuncs(const orc_params *p)
{
    if (p->kind == 0) return p->b * p->r;
    return p->b * ((p->r + 1) / 2);
}

/* Hash parameters of Algorithm 1's single_hash, drawn from SplitMix64. */
void orc_hash_params(const orc_params *p, uint64_t *a, uint64_t *bb)
{
    uint32_t F = orc_nfuncs(p);
    for (uint32_t f = 0; f < F; f++) {
        a[f] = orc_sm64(p->seed, 2ULL * f) | 1ULL;
        bb[f] = orc_sm64(p->seed, 2ULL * f + 1);
    }
}

/* h_f(x): top 32 bits of the 64-bit affine map a*x + b (wrapping). */
uint32_t orc_h(uint64_t a, uint64_t b, uint32_t x)
{
    uint64_t y = a * (uint64_t)x + b;
    return (uint32_t)(y >> 32);
}

/* ------------------------------------------------------------------ */
/* 2. per-function minima / maxima (§6.1, §6.2, Algorithm 1)           */
/* ------------------------------------------------------------------ */

/* Minimum and maximum of h_f over one fingerprint's K set bits, for every f. */
static void orc_row_values(const orc_params *p, const uint64_t *a, const uint64_t *bb,
                           const uint16_t *row, uint32_t *mn, uint32_t *mx)
{
    uint32_t F = orc_nfuncs(p);
    for (uint32_t f = 0; f < F; f++) {
        uint32_t lo = 0xFFFFFFFFu, hi = 0;
        for (uint32_t k = 0; k < p->K; k++) {
            uint32_t h = orc_h(a[f], bb[f], row[k]);
            if (h < lo) lo = h;
            if (h > hi) hi = h;
        }
        mn[f] = lo;
        if (mx) mx[f] = hi;
    }
}

/* mn[i*F + f] = min over the set bits x of fingerprint i of h_f(x);
 * mx likewise with max (written only when mx != NULL). */
void orc_values(const orc_params *p, const uint16_t *idx, uint64_t N, uint32_t ld,
                uint32_t *mn, uint32_t *mx)
{
    uint32_t F = orc_nfuncs(p);
    uint64_t *a = malloc(sizeof(uint64_t) * F), *bb = malloc(sizeof(uint64_t) * F);
    orc_hash_params(p, a, bb);
    for (uint64_t i = 0; i < N; i++)
        orc_row_values(p, a, bb, idx + i * (uint64_t)ld, mn + i * F, mx ? mx + i * F : NULL);
    free(a);
    free(bb);
}

/* ------------------------------------------------------------------ */
/* 3. bucket keys (Algorithm 1, hash_combine)                          */
/* ------------------------------------------------------------------ */

/* Fold the r band values of table t into one 32-bit key. */
static uint32_t orc_combine(const orc_params *p, uint32_t t, const uint32_t *mn_row,
                            const uint32_t *mx_row)
{
    uint32_t F = orc_nfuncs(p);
    uint64_t z = orc_sm64(p->seed, 2ULL * F + t);
    if (p->kind == 0) {
        for (uint32_t c = 0; c < p->r; c++) z = orc_mix64(z ^ (uint64_t)mn_row[t * p->r + c]);
    } else {
        uint32_t q = (p->r + 1) / 2;
        for (uint32_t c = 0; c < p->r; c++) {
            uint32_t f = t * q + c / 2;
            uint32_t w = (c % 2 == 0) ? mn_row[f] : mx_row[f];
            z = orc_mix64(z ^ (uint64_t)w);
        }
    }
    return (uint32_t)(z >> 32);
}

typedef struct {
    const orc_params *p;
    const uint16_t *idx;
    uint64_t N, i0, i1;
    uint32_t ld;
    uint32_t *keys;
} orc_keys_job;

static void *orc_keys_worker(void *arg)
{
    orc_keys_job *j = arg;
    const orc_params *p = j->p;
    uint32_t F = orc_nfuncs(p);
    uint32_t *mn = malloc(sizeof(uint32_t) * F), *mx = malloc(sizeof(uint32_t) * F);
    uint64_t *a = malloc(sizeof(uint64_t) * F), *bb = malloc(sizeof(uint64_t) * F);
    orc_hash_params(p, a, bb);
    for (uint64_t i = j->i0; i < j->i1; i++) {
        orc_row_values(p, a, bb, j->idx + i * (uint64_t)j->ld, mn, p->kind == 1 ? mx : NULL);
        for (uint32_t t = 0; t < p->b; t++) j->keys[(uint64_t)t * j->N + i] = orc_combine(p, t, mn, mx);
    }
    free(mn);
    free(mx);
    free(a);
    free(bb);
    return NULL;
}

static int orc_threads(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* keys[t*N + i] = bucket key of fingerprint i in table t (table-major).
 * Fingerprints are split over `nthreads` threads (the paper's parallel signature
 * generation, §6.4 "Parallelization"); every fingerprint is computed alone. */
int orc_keys(const orc_params *p, const uint16_t *idx, uint64_t N, uint32_t ld, uint32_t *keys,
             int nthreads)
{
    int T = orc_threads(nthreads);
    if ((uint64_t)T > N) T = N ? (int)N : 1;
    pthread_t *th = malloc(sizeof(pthread_t) * T);
    orc_keys_job *jobs = malloc(sizeof(orc_keys_job) * T);
    for (int k = 0; k < T; k++) {
        jobs[k] = (orc_keys_job){p, idx, N, N * k / T, N * (k + 1) / T, ld, keys};
        pthread_create(&th[k], NULL, orc_keys_worker, &jobs[k]);
    }
    for (int k = 0; k < T; k++) pthread_join(th[k], NULL);
    free(th);
    free(jobs);
    return T;
}

/* ------------------------------------------------------------------ */
/* 4. hash tables (§6.1 "Hash table construction")                     */
/* ------------------------------------------------------------------ */

static int orc_cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/* One table as (key, id) pairs ordered by key, then id: the canonical listing
 * of the table's buckets. */
void orc_table(const uint32_t *keys_t, uint64_t N, uint32_t *skey, uint32_t *sid)
{
    uint64_t *kv = malloc(sizeof(uint64_t) * (N ? N : 1));
    for (uint64_t i = 0; i < N; i++) kv[i] = ((uint64_t)keys_t[i] << 32) | i;
    qsort(kv, N, sizeof(uint64_t), orc_cmp_u64);
    for (uint64_t i = 0; i < N; i++) {
        skey[i] = (uint32_t)(kv[i] >> 32);
        sid[i] = (uint32_t)kv[i];
    }
    free(kv);
}

/* ------------------------------------------------------------------ */
/* 5. occurrence filter (§6.5 "Removing correlated noise")             */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_params *p;
    const uint32_t *keys;
    uint64_t N;
    uint32_t t0, t1;
    uint32_t *heavy_cnt; /* private per job: [N] */
} orc_drop_job;

static void *orc_drop_worker(void *arg)
{
    orc_drop_job *j = arg;
    uint64_t N = j->N;
    uint32_t *skey = malloc(sizeof(uint32_t) * (N ? N : 1));
    uint32_t *sid = malloc(sizeof(uint32_t) * (N ? N : 1));
    for (uint32_t t = j->t0; t < j->t1; t++) {
        orc_table(j->keys + (uint64_t)t * N, N, skey, sid);
        uint64_t s = 0;
        while (s < N) {
            uint64_t e = s + 1;
            while (e < N && skey[e] == skey[s]) e++;
            uint64_t size = e - s;
            if ((uint64_t)j->p->occ_den * size > (uint64_t)j->p->occ_num * N)
                for (uint64_t q = s; q < e; q++) j->heavy_cnt[sid[q]]++;
            s = e;
        }
    }
    free(skey);
    free(sid);
    return NULL;
}

/* heavy_cnt[i] = number of tables whose bucket holding i is heavy;
 * drop[i] = 2*heavy_cnt[i] > b.  Either output may be NULL. */
int orc_drop(const orc_params *p, const uint32_t *keys, uint64_t N, uint8_t *drop,
             uint32_t *heavy_cnt_out, int nthreads)
{
    uint32_t *cnt = calloc(N ? N : 1, sizeof(uint32_t));
    int T = orc_threads(nthreads);
    if (p->occ_num > 0 && N > 0) {
        if ((uint32_t)T > p->b) T = (int)p->b;
        pthread_t *th = malloc(sizeof(pthread_t) * T);
        orc_drop_job *jobs = malloc(sizeof(orc_drop_job) * T);
        for (int k = 0; k < T; k++) {
            jobs[k] = (orc_drop_job){p, keys, N, (uint32_t)((uint64_t)p->b * k / T),
                                     (uint32_t)((uint64_t)p->b * (k + 1) / T),
                                     calloc(N, sizeof(uint32_t))};
            pthread_create(&th[k], NULL, orc_drop_worker, &jobs[k]);
        }
        for (int k = 0; k < T; k++) {
            pthread_join(th[k], NULL);
            for (uint64_t i = 0; i < N; i++) cnt[i] += jobs[k].heavy_cnt[i];
            free(jobs[k].heavy_cnt);
        }
        free(th);
        free(jobs);
    } else {
        T = 1;
    }
    for (uint64_t i = 0; i < N; i++) {
        if (drop) drop[i] = (uint8_t)(2ULL * cnt[i] > p->b);
        if (heavy_cnt_out) heavy_cnt_out[i] = cnt[i];
    }
    free(cnt);
    return T;
}

/* ------------------------------------------------------------------ */
/* 6. search: votes per pair, threshold, canonical order                */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t n, cap;
    uint32_t *i, *j;
    uint8_t *votes;
} orc_list;

static void orc_list_push(orc_list *L, uint32_t i, uint32_t j, uint32_t votes)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->i = realloc(L->i, sizeof(uint32_t) * L->cap);
        L->j = realloc(L->j, sizeof(uint32_t) * L->cap);
        L->votes = realloc(L->votes, L->cap);
    }
    L->i[L->n] = i;
    L->j[L->n] = j;
    L->votes[L->n] = (uint8_t)votes;
    L->n++;
}

static int orc_pair_ok(const orc_params *p, const uint8_t *drop, uint64_t i, uint64_t j)
{
    if (drop && (drop[i] || drop[j])) return 0;
    return j > i && j - i > p->excl;
}

/* Bucket-wise search: every pair sharing a bucket in table t adds one vote
 * (§6.1 "Search").  Votes are collected as a list of (i, j) emissions that is
 * sorted and run-length counted -- the plainest exact count.
 * Returns the number of detections; the arrays are malloc'ed (orc_free). */
uint64_t orc_search(const orc_params *p, const uint32_t *keys, const uint8_t *drop, uint64_t N,
                    uint32_t **out_i, uint32_t **out_j, uint8_t **out_votes)
{
    uint64_t ne = 0, cap = 1024;
    uint64_t *em = malloc(sizeof(uint64_t) * cap);
    uint32_t *skey = malloc(sizeof(uint32_t) * (N ? N : 1));
    uint32_t *sid = malloc(sizeof(uint32_t) * (N ? N : 1));
    for (uint32_t t = 0; t < p->b; t++) {
        orc_table(keys + (uint64_t)t * N, N, skey, sid);
        uint64_t s = 0;
        while (s < N) {
            uint64_t e = s + 1;
            while (e < N && skey[e] == skey[s]) e++;
            for (uint64_t x = s; x < e; x++)
                for (uint64_t y = x + 1; y < e; y++) {
                    uint64_t i = sid[x], j = sid[y];
                    if (!orc_pair_ok(p, drop, i, j)) continue;
                    if (ne == cap) {
                        cap *= 2;
                        em = realloc(em, sizeof(uint64_t) * cap);
                    }
                    em[ne++] = (i << 32) | j;
                }
            s = e;
        }
    }
    free(skey);
    free(sid);
    qsort(em, ne, sizeof(uint64_t), orc_cmp_u64);
    orc_list L = {0};
    uint64_t s = 0;
    while (s < ne) {
        uint64_t e = s + 1;
        while (e < ne && em[e] == em[s]) e++;
        if (e - s >= p->v) orc_list_push(&L, (uint32_t)(em[s] >> 32), (uint32_t)em[s], (uint32_t)(e - s));
        s = e;
    }
    free(em);
    *out_i = L.i;
    *out_j = L.j;
    *out_votes = L.votes;
    return L.n;
}

/* Votes of one pair straight from the definition: tables with equal keys. */
uint32_t orc_pair_votes(const orc_params *p, const uint32_t *keys, uint64_t N, uint64_t i, uint64_t j)
{
    uint32_t votes = 0;
    for (uint32_t t = 0; t < p->b; t++) votes += keys[(uint64_t)t * N + i] == keys[(uint64_t)t * N + j];
    return votes;
}

/* Brute force over all pairs i < j (tiny inputs only). */
uint64_t orc_search_brute(const orc_params *p, const uint32_t *keys, const uint8_t *drop, uint64_t N,
                          uint32_t **out_i, uint32_t **out_j, uint8_t **out_votes)
{
    orc_list L = {0};
    for (uint64_t i = 0; i < N; i++)
        for (uint64_t j = i + 1; j < N; j++) {
            if (!orc_pair_ok(p, drop, i, j)) continue;
            uint32_t v = orc_pair_votes(p, keys, N, i, j);
            if (v >= p->v) orc_list_push(&L, (uint32_t)i, (uint32_t)j, v);
        }
    *out_i = L.i;
    *out_j = L.j;
    *out_votes = L.votes;
    return L.n;
}

/* Row i of the detection list: every j > i with its votes, from the
 * definition.  For sampled rows of inputs too large for orc_search. */
uint64_t orc_search_row(const orc_params *p, const uint32_t *keys, const uint8_t *drop, uint64_t N,
                        uint64_t i, uint32_t **out_j, uint8_t **out_votes)
{
    orc_list L = {0};
    for (uint64_t j = i + 1; j < N; j++) {
        if (!orc_pair_ok(p, drop, i, j)) continue;
        uint32_t v = orc_pair_votes(p, keys, N, i, j);
        if (v >= p->v) orc_list_push(&L, (uint32_t)i, (uint32_t)j, v);
    }
    free(L.i);
    *out_j = L.j;
    *out_votes = L.votes;
    return L.n;
}

void orc_free(void *ptr) { free(ptr); }

/* ------------------------------------------------------------------ */
/* 7. streaming replay (serving reading of §6.4 "Partition")           */
/* ------------------------------------------------------------------ */

/*
 * One streamed request, by definition.  keys [b][Ntot] holds the bucket keys
 * of every window of a station so far, in id order: the N0 history windows,
 * then all earlier requests' batches, then this request's batch [j0, Ntot).
 * A history window keeps its drop flag from the history alone (hist_drop,
 * orc_drop on the history keys).  Any later window w is dropped iff its key
 * falls in a heavy history bucket -- occ_den * size > occ_num * N0, size
 * counted over the N0 history windows -- in more than b/2 tables.
 * Reported: pairs (i, j), j in the batch, i < j, neither dropped,
 * j - i > E, votes >= v, sorted by (i, j).
 */
uint64_t orc_stream_query(const orc_params *p, const uint32_t *keys, uint64_t Ntot, uint64_t N0, uint64_t j0,
                          const uint8_t *hist_drop, uint32_t **out_i, uint32_t **out_j, uint8_t **out_votes)
{
    uint8_t *drop = calloc(Ntot ? Ntot : 1, 1);
    for (uint64_t w = 0; w < N0; w++) drop[w] = hist_drop ? hist_drop[w] : 0;
    if (p->occ_num > 0 && Ntot > N0) {
        uint32_t *cnt = calloc(Ntot - N0, sizeof(uint32_t));
        uint32_t *hk = malloc(sizeof(uint32_t) * (N0 ? N0 : 1));
        for (uint32_t t = 0; t < p->b; t++) {
            const uint32_t *kt = keys + (uint64_t)t * Ntot;
            for (uint64_t w = N0; w < Ntot; w++) {
                uint64_t size = 0; /* history windows sharing the key */
                for (uint64_t h = 0; h < N0; h++) size += kt[h] == kt[w];
                if ((uint64_t)p->occ_den * size > (uint64_t)p->occ_num * N0) cnt[w - N0]++;
            }
        }
        for (uint64_t w = N0; w < Ntot; w++) drop[w] = 2ULL * cnt[w - N0] > p->b;
        free(cnt);
        free(hk);
    }
    orc_list L = {0};
    for (uint64_t i = 0; i < Ntot; i++)
        for (uint64_t j = (i + 1 > j0 ? i + 1 : j0); j < Ntot; j++) {
            if (!orc_pair_ok(p, drop, i, j)) continue;
            uint32_t v = orc_pair_votes(p, keys, Ntot, i, j);
            if (v >= p->v) orc_list_push(&L, (uint32_t)i, (uint32_t)j, v);
        }
    free(drop);
    *out_i = L.i;
    *out_j = L.j;
    *out_votes = L.votes;
    return L.n;
}

/* ------------------------------------------------------------------ */
/* 8. channel level (§7.1 "Channel Level", §7.2 sort-merge-reduce)    */
/* ------------------------------------------------------------------ */

/*
 * The channels of one station see the same ground motion at the same times,
 * so their similarity matrices are summed and the sum is thresholded again.
 * The paper's procedure, in its order:
 *   sort    every channel's entries (dt = j - i, idx1 = i, sim) by dt, then idx1;
 *   merge   the sorted channel lists into one list in the same order (ties
 *           keep the channel order);
 *   reduce  consecutive entries with equal (dt, idx1) into one whose sim is
 *           their sum, discarding sums below thr.
 * Output: (i, j, summed sim) in (dt, idx1) order.  The sum of nch votes of at
 * most 255 each needs 16 bits.  Returns the number of entries; writes at most
 * cap of them.
 */
typedef struct {
    uint32_t dt, idx1, sim;
} orc_trip;

static int orc_cmp_trip(const void *x, const void *y)
{
    const orc_trip *a = x, *b = y;
    if (a->dt != b->dt) return a->dt < b->dt ? -1 : 1;
    if (a->idx1 != b->idx1) return a->idx1 < b->idx1 ? -1 : 1;
    return 0;
}

uint64_t orc_channel_merge(uint32_t nch, const uint64_t *M, const uint32_t *const *I, const uint32_t *const *J,
                           const uint8_t *const *V, uint32_t thr, uint32_t *out_i, uint32_t *out_j,
                           uint16_t *out_sim, uint64_t cap)
{
    /* sorting phase */
    orc_trip **ch = malloc(sizeof(orc_trip *) * (nch ? nch : 1));
    uint64_t *pos = calloc(nch ? nch : 1, sizeof(uint64_t));
    uint64_t total = 0;
    for (uint32_t c = 0; c < nch; c++) {
        ch[c] = malloc(sizeof(orc_trip) * (M[c] ? M[c] : 1));
        for (uint64_t k = 0; k < M[c]; k++) ch[c][k] = (orc_trip){J[c][k] - I[c][k], I[c][k], V[c][k]};
        qsort(ch[c], M[c], sizeof(orc_trip), orc_cmp_trip);
        total += M[c];
    }
    /* merging phase: repeatedly take the smallest head (the lowest channel on ties) */
    orc_trip *merged = malloc(sizeof(orc_trip) * (total ? total : 1));
    for (uint64_t k = 0; k < total; k++) {
        int best = -1;
        for (uint32_t c = 0; c < nch; c++) {
            if (pos[c] == M[c]) continue;
            if (best < 0 || orc_cmp_trip(&ch[c][pos[c]], &ch[best][pos[best]]) < 0) best = (int)c;
        }
        merged[k] = ch[best][pos[best]++];
    }
    /* reduce phase */
    uint64_t n = 0;
    for (uint64_t k = 0; k < total;) {
        uint64_t e = k;
        uint32_t sum = 0;
        while (e < total && merged[e].dt == merged[k].dt && merged[e].idx1 == merged[k].idx1) sum += merged[e++].sim;
        if (sum >= thr) {
            if (n < cap) {
                out_i[n] = merged[k].idx1;
                out_j[n] = merged[k].idx1 + merged[k].dt;
                out_sim[n] = (uint16_t)sum;
            }
            n++;
        }
        k = e;
    }
    for (uint32_t c = 0; c < nch; c++) free(ch[c]);
    free(ch);
    free(pos);
    free(merged);
    return n;
}

/* ------------------------------------------------------------------ */
/* 9. station level (§7.1 "Station Level", §7.2 "Station")             */
/* ------------------------------------------------------------------ */

/*
 * Thin diagonal clusters of one station's (combined) similarity matrix, in the
 * paper's steps:
 *   runs    along every diagonal dt, the maximal sequences of entries whose
 *           consecutive idx1 differ by less than `gap` (the largest gap inside
 *           a sequence is smaller than the gap parameter);
 *   merge   runs on adjacent diagonals (dt and dt + 1) are merged when their
 *           idx1 ranges come within `gap` of each other, as long as the merged
 *           cluster spans at most `width` diagonals (the paper's "relatively
 *           narrow width");
 *   summary per cluster: bounding box (dt_min, dt_max, idx1_min, idx1_max),
 *           number of entries and summed similarity;
 *   prune   clusters of fewer than `min_n` entries (min_n = 2 drops isolated
 *           matches).
 * Readings (the paper leaves them open): the merge is greedy in (dt, idx1)
 * order of the runs -- each run, taken in that order, joins the first cluster
 * of the previous diagonal that it comes within `gap` of and that the width
 * limit lets it join; clusters are reported in (dt_min, idx1_min) order;
 * gap >= 1.
 * Input: n entries (i, j, sim) in (dt, idx1) order, dt = j - i, idx1 = i.
 * Output: 6 uint64 per cluster (dt_min, dt_max, idx1_min, idx1_max, count, sim);
 * returns the number of clusters, writes at most cap.
 */
typedef struct {
    uint64_t dt, s, e, n, sim; /* one run: diagonal, idx1 range, entries, summed sim */
    int64_t parent;            /* union-find over runs */
    uint64_t dt_min, dt_max, s_min, e_max; /* the cluster's box (valid at roots) */
} orc_run;

static int64_t orc_root(orc_run *r, int64_t x)
{
    while (r[x].parent != x) {
        r[x].parent = r[r[x].parent].parent;
        x = r[x].parent;
    }
    return x;
}

static int orc_cmp_box(const void *x, const void *y)
{
    const uint64_t *a = x, *b = y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[2] != b[2]) return a[2] < b[2] ? -1 : 1;
    return 0;
}

uint64_t orc_station_clusters(const uint32_t *I, const uint32_t *J, const uint16_t *S, uint64_t n, uint32_t gap,
                              uint32_t width, uint32_t min_n, uint64_t *out, uint64_t cap)
{
    /* runs along each diagonal */
    orc_run *r = malloc(sizeof(orc_run) * (n ? n : 1));
    uint64_t nr = 0;
    for (uint64_t k = 0; k < n;) {
        const uint64_t dt = J[k] - I[k];
        orc_run run = {dt, I[k], I[k], 0, 0, 0, 0, 0, 0, 0};
        uint64_t e = k;
        while (e < n && J[e] - I[e] == dt && (e == k || I[e] - I[e - 1] < gap)) {
            run.e = I[e];
            run.n++;
            run.sim += S[e];
            e++;
        }
        run.parent = (int64_t)nr;
        run.dt_min = run.dt_max = dt;
        run.s_min = run.s;
        run.e_max = run.e;
        r[nr++] = run;
        k = e;
    }
    /* merge across adjacent diagonals, runs in (dt, idx1) order */
    uint64_t prev0 = 0; /* first run of diagonal dt - 1 */
    for (uint64_t x = 0; x < nr; x++) {
        if (x > 0 && r[x].dt != r[x - 1].dt) {
            /* the runs of the previous diagonal start where that diagonal started */
            uint64_t y = x - 1;
            while (y > 0 && r[y - 1].dt == r[x - 1].dt) y--;
            prev0 = y;
        }
        if (x == 0 || r[prev0].dt + 1 != r[x].dt) continue;
        for (uint64_t y = prev0; y < nr && r[y].dt == r[x].dt - 1; y++) {
            const int near = r[y].s <= r[x].e + gap - 1 && r[x].s <= r[y].e + gap - 1;
            if (!near) continue;
            const int64_t a = orc_root(r, (int64_t)y), b = orc_root(r, (int64_t)x);
            if (a == b) continue;
            const uint64_t lo = r[a].dt_min < r[b].dt_min ? r[a].dt_min : r[b].dt_min;
            const uint64_t hi = r[a].dt_max > r[b].dt_max ? r[a].dt_max : r[b].dt_max;
            if (hi - lo + 1 > width) continue;
            r[b].parent = a; /* x's cluster joins the earlier one */
            r[a].dt_min = lo;
            r[a].dt_max = hi;
            if (r[b].s_min < r[a].s_min) r[a].s_min = r[b].s_min;
            if (r[b].e_max > r[a].e_max) r[a].e_max = r[b].e_max;
            r[a].n += r[b].n;
            r[a].sim += r[b].sim;
            break; /* the first cluster it comes near */
        }
    }
    /* summaries of the roots, pruned, in (dt_min, idx1_min) order */
    uint64_t *box = malloc(sizeof(uint64_t) * 6 * (nr ? nr : 1));
    uint64_t nc = 0;
    for (uint64_t x = 0; x < nr; x++) {
        if (r[x].parent != (int64_t)x || r[x].n < min_n) continue;
        uint64_t *b = box + 6 * nc++;
        b[0] = r[x].dt_min;
        b[1] = r[x].dt_max;
        b[2] = r[x].s_min;
        b[3] = r[x].e_max;
        b[4] = r[x].n;
        b[5] = r[x].sim;
    }
    qsort(box, nc, sizeof(uint64_t) * 6, orc_cmp_box);
    for (uint64_t c = 0; c < nc && c < cap; c++) memcpy(out + 6 * c, box + 6 * c, sizeof(uint64_t) * 6);
    free(box);
    free(r);
    return nc;
}
