/*
 * gen.c -- seeded synthetic fingerprint workloads.
 *
 * Stands in for the continuous-data fingerprints of the paper's GeoNet and
 * NCEDC stations (§8 "Dataset"), which are not available here.  A fingerprint
 * is a binary vector of D bits with exactly K set bits (§5.1, "Binarize";
 * top-K coefficients), stored as an ascending uint16 index list.
 *
 * This module is the ONE input source shared by the CUDA path and the oracle.
 * It holds none of the search method's arithmetic: it only draws sets.
 *
 * Structure of a station's N windows (1 window = 1 s lag, §6.4 "Partition"):
 *   1. every window starts as a uniform random K-subset of [0, D);
 *   2. each periodic noise source p (period P_p windows) has a base set and a
 *      random phase; every window phase + k*P_p becomes a noisy copy of it
 *      (repeating non-seismic signals, §6.5 "Removing correlated noise");
 *   3. each template tau (a repeating earthquake source, §1) has a base set and
 *      U{rep_lo..rep_hi} repeats at uniform random windows, each a noisy copy.
 *   Later steps overwrite earlier ones at the same window.
 * A noisy copy with re-draw fraction x removes round(x*K) uniformly chosen set
 * bits and adds as many uniform bits from D minus the remaining set, so
 * exactly K bits stay set.
 *
 * Randomness is counter based (SplitMix64, Steele, Lea & Flood 2014): every
 * draw is a pure function of (seed, stream, counter), so rows are generated
 * independently and in parallel, identically on every machine.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define SYN_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t syn_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Stream key for (seed, domain, id); draws are syn_mix(key + (n+1)*GAMMA). */
static uint64_t syn_stream(uint64_t seed, uint64_t domain, uint64_t id)
{
    return syn_mix(syn_mix(seed ^ (domain * 0xD1B54A32D192ED03ULL)) + (id + 1) * SYN_GAMMA);
}

typedef struct {
    uint64_t key, n;
} syn_rng;

static uint64_t syn_next(syn_rng *g)
{
    g->n++;
    return syn_mix(g->key + g->n * SYN_GAMMA);
}

/* Uniform integer in [0, m) by the multiply-high method. */
static uint64_t syn_below(syn_rng *g, uint64_t m)
{
    return (uint64_t)(((unsigned __int128)syn_next(g) * m) >> 64);
}

enum { DOM_ROW = 1, DOM_PBASE = 2, DOM_PPHASE = 3, DOM_TBASE = 4, DOM_TPLACE = 5, DOM_NOISE = 6,
       DOM_TOFF = 7, DOM_SKEW = 8 };

/*
 * Optional imbalance of the bits (the paper's observation that some
 * fingerprint elements are non-zero far more often than others, and that
 * some co-occur, §6.3 "Cause of hash collisions"): bit x has weight
 * (1 + rank(x))^-skew, ranks a random permutation of [0, D) drawn from the
 * station seed; after a bit is drawn, its partner -- the bit of the
 * neighbouring rank, rank ^ 1 -- is also set with probability corr.
 * skew = corr = 0 is the uniform generator, draw for draw.
 */
typedef struct {
    const double *cdf;    /* cdf[r] = total weight of ranks 0..r; NULL = uniform */
    const uint16_t *bit;  /* bit of rank r */
    const uint16_t *rank; /* rank of bit x */
    double corr;
} syn_skew;

#define OWNER_RANDOM 0u
#define OWNER_PERIODIC (1u << 30)
#define OWNER_TEMPLATE (2u << 30)

/* Writes the ascending list of the bits set in bitmap `bm` (D bits) to out. */
static uint32_t syn_emit(const uint64_t *bm, uint32_t D, uint16_t *out)
{
    uint32_t n = 0;
    for (uint32_t w = 0; w < (D + 63) / 64; w++) {
        uint64_t x = bm[w];
        while (x) {
            out[n++] = (uint16_t)(w * 64 + (uint32_t)__builtin_ctzll(x));
            x &= x - 1;
        }
    }
    return n;
}

/* One bit: uniform on [0, D), or by the skew weights. */
static uint32_t syn_draw(syn_rng *g, const syn_skew *sk, uint32_t D)
{
    if (!sk || !sk->cdf) return (uint32_t)syn_below(g, D);
    const double u = (double)(syn_next(g) >> 11) * (1.0 / 9007199254740992.0) * sk->cdf[D - 1];
    uint32_t lo = 0, hi = D - 1; /* first rank whose cumulative weight exceeds u */
    while (lo < hi) {
        const uint32_t m = (lo + hi) / 2;
        if (sk->cdf[m] > u) hi = m;
        else lo = m + 1;
    }
    return sk->bit[lo];
}

/* Sets bit x unless set; with skew and corr > 0 also, at probability corr,
 * its partner (while fewer than `want` bits are set).  Returns the bits added. */
static uint32_t syn_take(syn_rng *g, const syn_skew *sk, uint32_t D, uint64_t *bm, uint32_t x, uint32_t have,
                         uint32_t want)
{
    if (bm[x >> 6] >> (x & 63) & 1) return 0;
    bm[x >> 6] |= 1ULL << (x & 63);
    uint32_t added = 1;
    if (sk && sk->cdf && sk->corr > 0 && have + 1 < want) {
        const double c = (double)(syn_next(g) >> 11) * (1.0 / 9007199254740992.0);
        const uint32_t r = sk->rank[x] ^ 1u;
        if (c < sk->corr && r < D) {
            const uint32_t y = sk->bit[r];
            if (!(bm[y >> 6] >> (y & 63) & 1)) {
                bm[y >> 6] |= 1ULL << (y & 63);
                added++;
            }
        }
    }
    return added;
}

/* Random K-subset of [0, D) (uniform, or by the skew), ascending. */
static void syn_subset(syn_rng *g, const syn_skew *sk, uint32_t D, uint32_t K, uint64_t *bm, uint16_t *out)
{
    memset(bm, 0, sizeof(uint64_t) * ((D + 63) / 64));
    uint32_t have = 0;
    while (have < K) have += syn_take(g, sk, D, bm, syn_draw(g, sk, D), have, K);
    syn_emit(bm, D, out);
}

/* Noisy copy of the ascending K-set `base`: remove m = round(x*K) uniformly
 * chosen members, then add m uniform bits of D outside the remaining set. */
static void syn_copy(syn_rng *g, const syn_skew *sk, const uint16_t *base, uint32_t D, uint32_t K, double x,
                     uint64_t *bm, uint32_t *perm, uint16_t *out)
{
    uint32_t m = (uint32_t)(x * K + 0.5);
    if (m > K) m = K;
    for (uint32_t k = 0; k < K; k++) perm[k] = k;
    for (uint32_t k = 0; k < m; k++) { /* partial Fisher-Yates: perm[0..m) removed */
        uint32_t s = k + (uint32_t)syn_below(g, K - k);
        uint32_t tmp = perm[k];
        perm[k] = perm[s];
        perm[s] = tmp;
    }
    memset(bm, 0, sizeof(uint64_t) * ((D + 63) / 64));
    for (uint32_t k = m; k < K; k++) bm[base[perm[k]] >> 6] |= 1ULL << (base[perm[k]] & 63);
    /* the removed bits may come back: D minus the *remaining* set is eligible */
    uint32_t added = 0;
    while (added < m) added += syn_take(g, sk, D, bm, syn_draw(g, sk, D), added, m);
    syn_emit(bm, D, out);
}

typedef struct {
    uint64_t N, w0, w1, row0, seed;
    uint32_t D, K, ld;
    uint16_t *out;
    const uint32_t *owner; /* indexed by w - row0 */
    const uint64_t *ids;   /* when set: row w - row0 is window ids[w - row0] */
    const uint16_t *pbase, *tbase;
    double per_redraw, tpl_redraw;
    const syn_skew *sk;
} syn_job;

static void *syn_worker(void *arg)
{
    syn_job *j = arg;
    uint64_t *bm = malloc(sizeof(uint64_t) * ((j->D + 63) / 64));
    uint32_t *perm = malloc(sizeof(uint32_t) * (j->K ? j->K : 1));
    for (uint64_t r = j->w0; r < j->w1; r++) {
        const uint64_t w = j->ids ? j->ids[r - j->row0] : r; /* the window drawn into row r - row0 */
        uint16_t *row = j->out + (r - j->row0) * (uint64_t)j->ld;
        uint32_t own = j->owner[r - j->row0];
        uint32_t kind = own & (3u << 30), id = own & ((1u << 30) - 1);
        if (kind == OWNER_RANDOM) {
            syn_rng g = {syn_stream(j->seed, DOM_ROW, w), 0};
            syn_subset(&g, j->sk, j->D, j->K, bm, row);
        } else {
            syn_rng g = {syn_stream(j->seed, DOM_NOISE, w), 0};
            if (kind == OWNER_PERIODIC)
                syn_copy(&g, j->sk, j->pbase + (uint64_t)id * j->K, j->D, j->K, j->per_redraw, bm, perm, row);
            else
                syn_copy(&g, j->sk, j->tbase + (uint64_t)id * j->K, j->D, j->K, j->tpl_redraw, bm, perm, row);
        }
        for (uint32_t k = j->K; k < j->ld; k++) row[k] = 0xFFFF; /* row padding */
    }
    free(bm);
    free(perm);
    return NULL;
}

/*
 * Fills out[nrows][ld] (ld >= K; out == NULL: no rows, owners only) with
 * windows row0 .. row0 + nrows - 1 of the
 * station's N windows and, when owner_out != NULL, owner_out[nrows] with each
 * window's source: 0 random, (1<<30)|p periodic source p, (2<<30)|tau
 * template tau.  Every window depends only on (seed, its index), so any range
 * of rows is drawn exactly as in the whole station (rows of a large station
 * can be drawn chunk by chunk).
 *
 * Templates draw their base sets and repeat counts from `tpl_seed` (shared
 * by all stations of a network) and their repeat windows uniformly from
 * [0, place_range); a station adds its own offset U{0..tpl_offset_max} per
 * template (drawn from `seed`) and keeps the repeats that land inside [0, N).
 * Periodic sources and everything else draw from `seed`.
 * Returns the number of threads used, or -1 on bad arguments.
 */
static int syn_cmp_u64(const void *a, const void *b)
{
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* position of w among the sorted distinct ids sid[0 .. m), or -1 */
static int64_t syn_find(const uint64_t *sid, uint64_t m, uint64_t w)
{
    uint64_t lo = 0, hi = m;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (sid[mid] < w) lo = mid + 1;
        else hi = mid;
    }
    return lo < m && sid[lo] == w ? (int64_t)lo : -1;
}

/* rows row0 .. row0 + nrows - 1, or (ids != NULL) the windows ids[0 .. nrows) */
static int syn_generate(uint64_t N, uint64_t row0, uint64_t nrows, const uint64_t *ids, uint32_t D, uint32_t K,
                        uint16_t *out, uint32_t ld, uint64_t seed, uint32_t n_periodic, const uint64_t *periods,
                        double per_redraw, uint32_t n_templates, uint32_t rep_lo, uint32_t rep_hi,
                        double tpl_redraw, uint64_t tpl_seed, uint64_t place_range, uint32_t tpl_offset_max,
                        int nthreads, uint32_t *owner_out, double skew, double corr)
{
    if (D == 0 || D > 65536 || K == 0 || K > D || ld < K || rep_hi < rep_lo) return -1;
    if (!ids && (row0 > N || nrows > N - row0)) return -1;
    uint64_t *sid = NULL, m = 0; /* the listed windows, sorted and distinct */
    if (ids) {
        for (uint64_t k = 0; k < nrows; k++)
            if (ids[k] >= N) return -1;
        sid = malloc(sizeof(uint64_t) * (nrows ? nrows : 1));
        memcpy(sid, ids, sizeof(uint64_t) * nrows);
        qsort(sid, nrows, sizeof(uint64_t), syn_cmp_u64);
        for (uint64_t k = 0; k < nrows; k++)
            if (m == 0 || sid[m - 1] != sid[k]) sid[m++] = sid[k];
        row0 = 0;
    }
    if (!(skew >= 0) || !(corr >= 0 && corr <= 1)) return -1;
    /* the skew: ranks drawn from the station seed (a Fisher-Yates shuffle) */
    syn_skew skv = {NULL, NULL, NULL, corr};
    double *cdf = NULL;
    uint16_t *sbit = NULL, *srank = NULL;
    if (skew > 0) {
        cdf = malloc(sizeof(double) * D);
        sbit = malloc(sizeof(uint16_t) * D);
        srank = malloc(sizeof(uint16_t) * D);
        for (uint32_t x = 0; x < D; x++) sbit[x] = (uint16_t)x;
        syn_rng q = {syn_stream(seed, DOM_SKEW, 0), 0};
        for (uint32_t x = D - 1; x > 0; x--) {
            const uint32_t y = (uint32_t)syn_below(&q, (uint64_t)x + 1);
            const uint16_t t = sbit[x];
            sbit[x] = sbit[y];
            sbit[y] = t;
        }
        double acc = 0;
        for (uint32_t r = 0; r < D; r++) {
            acc += pow(1.0 + r, -skew);
            cdf[r] = acc;
            srank[sbit[r]] = (uint16_t)r;
        }
        skv.cdf = cdf;
        skv.bit = sbit;
        skv.rank = srank;
    }
    const syn_skew *sk = skew > 0 ? &skv : NULL;
    const int rows_wanted = out != NULL; /* out == NULL: owner codes only */
    if (place_range == 0) place_range = N;
    const uint64_t row1 = row0 + nrows;
    uint32_t *owner = owner_out ? owner_out : malloc(sizeof(uint32_t) * (nrows ? nrows : 1));
    memset(owner, 0, sizeof(uint32_t) * nrows);
    uint32_t *down = ids ? calloc(m ? m : 1, sizeof(uint32_t)) : NULL; /* owner of each distinct id */
    uint64_t *bm = malloc(sizeof(uint64_t) * ((D + 63) / 64));

    uint16_t *pbase = malloc(sizeof(uint16_t) * (uint64_t)K * (n_periodic ? n_periodic : 1));
    for (uint32_t p = 0; p < n_periodic; p++) {
        syn_rng g = {syn_stream(seed, DOM_PBASE, p), 0};
        syn_subset(&g, sk, D, K, bm, pbase + (uint64_t)p * K);
        syn_rng h = {syn_stream(seed, DOM_PPHASE, p), 0};
        uint64_t P = periods[p] ? periods[p] : 1;
        uint64_t w = syn_below(&h, P);
        if (ids) {
            for (uint64_t k = 0; k < m; k++)
                if (sid[k] >= w && (sid[k] - w) % P == 0) down[k] = OWNER_PERIODIC | p;
            continue;
        }
        if (w < row0) w += (row0 - w + P - 1) / P * P; /* first copy at or after row0 */
        for (; w < row1; w += P) owner[w - row0] = OWNER_PERIODIC | p;
    }

    uint16_t *tbase = malloc(sizeof(uint16_t) * (uint64_t)K * (n_templates ? n_templates : 1));
    for (uint32_t t = 0; t < n_templates; t++) {
        syn_rng g = {syn_stream(tpl_seed, DOM_TBASE, t), 0};
        syn_subset(&g, sk, D, K, bm, tbase + (uint64_t)t * K);
        syn_rng pl = {syn_stream(tpl_seed, DOM_TPLACE, t), 0};
        uint32_t reps = rep_lo + (uint32_t)syn_below(&pl, (uint64_t)(rep_hi - rep_lo) + 1);
        syn_rng off = {syn_stream(seed, DOM_TOFF, t), 0};
        uint64_t delta = syn_below(&off, (uint64_t)tpl_offset_max + 1);
        for (uint32_t k = 0; k < reps; k++) {
            uint64_t w = syn_below(&pl, place_range) + delta;
            if (ids) {
                const int64_t q = w < N ? syn_find(sid, m, w) : -1;
                if (q >= 0) down[q] = OWNER_TEMPLATE | t;
            } else if (w < N && w >= row0 && w < row1) {
                owner[w - row0] = OWNER_TEMPLATE | t;
            }
        }
    }
    free(bm);
    if (ids)
        for (uint64_t k = 0; k < nrows; k++) owner[k] = down[syn_find(sid, m, ids[k])];

    int T = nthreads;
    if (T <= 0) {
        long n = sysconf(_SC_NPROCESSORS_ONLN);
        T = n > 0 ? (int)n : 1;
    }
    if ((uint64_t)T > nrows / 4096 + 1) T = (int)(nrows / 4096 + 1);
    if (!rows_wanted) T = 0;
    pthread_t *th = malloc(sizeof(pthread_t) * (T ? T : 1));
    syn_job *jobs = malloc(sizeof(syn_job) * (T ? T : 1));
    for (int k = 0; k < T; k++) {
        jobs[k] = (syn_job){N,   row0 + nrows * k / T, row0 + nrows * (k + 1) / T, row0, seed, D, K, ld,
                            out, owner, ids, pbase, tbase, per_redraw, tpl_redraw, sk};
        pthread_create(&th[k], NULL, syn_worker, &jobs[k]);
    }
    for (int k = 0; k < T; k++) pthread_join(th[k], NULL);
    free(th);
    free(jobs);
    free(pbase);
    free(tbase);
    free(cdf);
    free(sbit);
    free(srank);
    free(down);
    free(sid);
    if (!owner_out) free(owner);
    return T;
}

/*
 * Fills out[nrows][ld] (ld >= K; out == NULL: owners only) with windows
 * row0 .. row0 + nrows - 1 of the station's N windows; see syn_generate.
 */
int synth_generate_rows(uint64_t N, uint64_t row0, uint64_t nrows, uint32_t D, uint32_t K, uint16_t *out,
                        uint32_t ld, uint64_t seed, uint32_t n_periodic, const uint64_t *periods,
                        double per_redraw, uint32_t n_templates, uint32_t rep_lo, uint32_t rep_hi,
                        double tpl_redraw, uint64_t tpl_seed, uint64_t place_range, uint32_t tpl_offset_max,
                        int nthreads, uint32_t *owner_out, double skew, double corr)
{
    return syn_generate(N, row0, nrows, NULL, D, K, out, ld, seed, n_periodic, periods, per_redraw, n_templates,
                        rep_lo, rep_hi, tpl_redraw, tpl_seed, place_range, tpl_offset_max, nthreads, owner_out, skew,
                        corr);
}

/*
 * Windows ids[0 .. n) of the station (any order, repeats allowed) into
 * out[n][ld], each exactly the row the whole station has (owners as well,
 * when owner_out != NULL); the sources' placements are walked once for all
 * of them.
 */
int synth_generate_ids(uint64_t N, const uint64_t *ids, uint64_t n, uint32_t D, uint32_t K, uint16_t *out,
                       uint32_t ld, uint64_t seed, uint32_t n_periodic, const uint64_t *periods, double per_redraw,
                       uint32_t n_templates, uint32_t rep_lo, uint32_t rep_hi, double tpl_redraw, uint64_t tpl_seed,
                       uint64_t place_range, uint32_t tpl_offset_max, int nthreads, uint32_t *owner_out,
                       double skew, double corr)
{
    return syn_generate(N, 0, n, ids, D, K, out, ld, seed, n_periodic, periods, per_redraw, n_templates, rep_lo,
                        rep_hi, tpl_redraw, tpl_seed, place_range, tpl_offset_max, nthreads, owner_out, skew, corr);
}

/* The whole station: rows 0 .. N - 1 (see synth_generate_rows). */
int synth_generate(uint64_t N, uint32_t D, uint32_t K, uint16_t *out, uint32_t ld, uint64_t seed,
                   uint32_t n_periodic, const uint64_t *periods, double per_redraw,
                   uint32_t n_templates, uint32_t rep_lo, uint32_t rep_hi, double tpl_redraw,
                   uint64_t tpl_seed, uint64_t place_range, uint32_t tpl_offset_max,
                   int nthreads, uint32_t *owner_out)
{
    return synth_generate_rows(N, 0, N, D, K, out, ld, seed, n_periodic, periods, per_redraw, n_templates, rep_lo,
                               rep_hi, tpl_redraw, tpl_seed, place_range, tpl_offset_max, nthreads, owner_out, 0.0,
                               0.0);
}
