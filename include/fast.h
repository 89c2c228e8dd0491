/*
 * fast.h -- C-ABI of the GB300 LSH similarity search over binary waveform
 * fingerprints (Rong et al., "Locality-Sensitive Hashing for Earthquake
 * Detection: A Case Study of Scaling Data-Driven Science", §6).
 *
 * Problem (§6.1): given N binary fingerprints (one per time window, §5.1),
 * find every pair (i, j), i < j, that shares a hash bucket in at least v of
 * b independent hash tables, where each table keys a fingerprint by r
 * MinHash (or Min-Max hash, §6.2) values.  Pairs of nearby windows
 * (j - i <= excl) are excluded as self-matches (§7.1 "Station Level"), and
 * fingerprints caught by the occurrence filter (§6.5) take part in no pair.
 * Each detection is reported as (i, j, votes); in the paper's triplet form
 * (§7.2) that is (dt = j - i, idx1 = i, sim = votes).
 *
 * Conventions for every call:
 *   - Pointers named d_* are device pointers on the context's device; h_*
 *     are host pointers (pinned memory is faster but not required).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; device inputs must stay valid until
 *     the stream reaches the call's work.
 *   - Every call returns fast_status and never aborts.  Invalid arguments are
 *     reported as FAST_EINVAL before any work is enqueued; invalid data found
 *     on the device (an index >= D) is reported by the call that synchronises
 *     on it.  fast_last_error() gives a human-readable message.
 *   - Objects returned through out-pointers (tables, results) are owned by the
 *     caller and must be released with the matching *_free; they must not
 *     outlive the context that made them.
 *   - There is no CPU fallback: without a usable CUDA device every call fails
 *     with FAST_ECUDA.
 */
#ifndef FAST_H
#define FAST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FAST_OK = 0,
    FAST_EINVAL = 1,    /* bad argument or bad input data                     */
    FAST_ENOMEM = 2,    /* device allocation failed                            */
    FAST_EBUDGET = 3,   /* the work does not fit the context's HBM budget      */
    FAST_EMAPFULL = 4,  /* a device hash map ran past its probe limit          */
    FAST_ETIMEOUT = 5,  /* a bounded wait ran out                              */
    FAST_EPENDING = 6,  /* a streamed request is not finished yet              */
    FAST_ECUDA = 7,     /* a CUDA runtime call failed                          */
    FAST_EINTERNAL = 8  /* broken internal invariant (a bug)                   */
} fast_status;

typedef enum {
    FAST_MINHASH = 0, /* §6.1: r minima per table, F = b*r functions                  */
    FAST_MINMAX = 1   /* §6.2: min and max per function, F = b*ceil(r/2) functions    */
} fast_hash_kind;

/*
 * Search parameters.  Paper notation (§6.3): t = b tables, k = r values per
 * table, m = v matches.
 *   D, K      fingerprint dimension and set bits per fingerprint (§5.1);
 *             1 <= K <= D <= 65536.
 *   b, r      tables and values per table; 1 <= b <= 255, 1 <= r <= 16.
 *   kind      fast_hash_kind.
 *   seed      hash seed: the F hash functions h_f(x) = high32(a_f*x + b_f)
 *             take a_f = sm64(seed, 2f) | 1 and b_f = sm64(seed, 2f+1), where
 *             sm64(s, n) is the n-th SplitMix64 output of seed s; the bucket
 *             key of table t folds its r values w into z = sm64(seed, 2F+t)
 *             by z = mix64(z ^ w) and keeps high32(z) (Algorithm 1,
 *             hash_combine, with the hash family fixed by this library).
 *   v         report a pair when it shares a bucket in >= v tables; 1 <= v <= b.
 *   excl      report a pair only when j - i > excl.
 *   occ_num, occ_den
 *             occurrence filter (§6.5), static form: a bucket is heavy when
 *             occ_den * size > occ_num * N; a fingerprint in heavy buckets in
 *             more than b/2 tables is dropped.  occ_num = 0 turns it off.
 *   table_group
 *             tables sorted at once by the table build (0 = all b; at most
 *             b): the tables are radix-sorted table_group at a time straight
 *             into the table set, so the sort's scratch holds table_group * N
 *             (key, id) pairs instead of b * N.  The table set itself keeps
 *             all b tables, and the search counts votes over all of them, so
 *             the result does not depend on the value (§6.4 "Partition":
 *             identical results).
 *   query_part
 *             query partitions of the pair buffer (0 = automatic: as many as
 *             the memory left needs); identical results for any value (§6.4).
 */
typedef struct {
    uint32_t D, K, b, r;
    uint32_t kind;
    uint64_t seed;
    uint32_t v, excl;
    uint32_t occ_num, occ_den;
    uint32_t table_group;
    uint32_t query_part;
} fast_params;

typedef struct fast_ctx fast_ctx;
typedef struct fast_tables fast_tables;
typedef struct fast_result fast_result;

/*
 * Per-stage device times (ms, CUDA events on the call's stream) and counters
 * of the most recent fast_detect / fast_search on a context.
 */
typedef struct {
    float ms_sig, ms_sort, ms_filter, ms_enum, ms_dense, ms_sparse, ms_output, ms_total;
    uint64_t n_fingerprints;  /* N                                                  */
    uint64_t n_dropped;       /* fingerprints removed by the occurrence filter      */
    uint64_t n_emissions;     /* sparse bucket pairs counted in the vote map         */
    uint64_t n_dense_pairs;   /* pairs compared directly inside dense groups         */
    uint64_t n_groups;        /* dense groups (components of large buckets)          */
    uint64_t n_detections;    /* M                                                   */
    uint64_t map_slots;       /* vote-map capacity (slots) of the last partition     */
    uint64_t n_launches;      /* CUDA kernels launched by the call                   */
    uint64_t n_long_rows;     /* rows of row groups too large for one shared-memory
                                 hash, voted one CTA per row                          */
    uint64_t n_huge_rows;     /* long rows whose hash lives in global scratch         */
    uint64_t max_row;         /* most candidates of one long row                      */
    uint32_t query_parts;     /* query partitions actually used                      */
    uint32_t sort_passes;     /* radix passes per table sort                         */
    /* the sparse stage of the row-partitioned search, split: counting the
       small/medium-bucket pairs per row group, writing them, voting */
    float ms_pair_count, ms_pair_emit, ms_vote;
    /* single kernels inside those, summed over the query partitions: the
       small-bucket pair writer, the warp-per-group vote */
    float ms_k_pairs, ms_k_vote;
    uint64_t n_pairs_small;   /* of n_emissions: pairs of buckets with at most 32 entries */
    uint64_t peak_bytes;      /* most device memory held at once during the call    */
    uint64_t n_overflow;      /* single-pass pairs past their group's region slots   */
    uint64_t max_group;       /* members of the largest dense group                  */
    /* more single kernels of the sparse stage (ms, summed over the query
       partitions): the medium-bucket pair writer, the block-level votes
       (groups and rows too large for a warp), and, when pairs are counted
       before they are written, the two counting kernels */
    float ms_k_medium, ms_k_vote_block, ms_k_count_small, ms_k_count_medium;
    uint32_t dense_fallback;  /* 1 when the cluster-mask scratch did not fit and every
                                 dense group was voted by direct key comparison   */
    uint32_t large_min;       /* the dense-group threshold the search used (a batch
                                 with the automatic threshold: its largest station
                                 threshold)                                         */
    uint32_t group_shift;     /* sparse row groups hold 2^group_shift rows           */
    uint32_t region_slots;    /* single-pass slots per row group (0: pairs counted
                                 first, then written)                               */
} fast_stats;

/*
 * Creates a context on the current CUDA device: validates `p`, draws the
 * hash parameters and builds the per-function rank tables used by fast_sig.
 * hbm_budget_bytes bounds the device memory the context and the objects it
 * returns may hold at once (0 = no bound).  *out is NULL on failure.
 */
fast_status fast_create(const fast_params *p, uint64_t hbm_budget_bytes, fast_ctx **out);

/* Releases the context and its workspace.  NULL is a no-op. */
void fast_destroy(fast_ctx *ctx);

/* Message of the last failure on `ctx` (never NULL; "" after success). */
const char *fast_last_error(const fast_ctx *ctx);

/*
 * Signature generation (§6.1 "Hash signature generation", §6.2 Min-Max hash,
 * Algorithm 1).  d_idx: N rows of ld >= K uint16 set-bit indices (row i at
 * d_idx + i*ld; order within a row does not matter; entries K..ld-1 are
 * ignored).  Writes d_sig[t*N + i] = bucket key of fingerprint i in table t
 * (table-major, b*N uint32, caller-allocated).  An index >= D makes the call
 * fail with FAST_EINVAL when it synchronises (fast_sig synchronises `stream`).
 */
fast_status fast_sig(fast_ctx *ctx, const uint16_t *d_idx, uint64_t N, uint32_t ld, uint32_t *d_sig,
                     void *stream);

/*
 * Signatures of a station too large to hold its fingerprints in device
 * memory at once (§6.1 "Hash signature generation", Algorithm 1; §6.4
 * "Partition"), fed in chunks: d_idx holds n rows (ld >= K uint16 each) that
 * are windows col0 .. col0 + n - 1 of a station of N windows; their keys go
 * to d_sig[t*N + col0 + k] of the caller's [b][N] key array (caller-allocated,
 * device).  col0 + n <= N.  Enqueues the work on `stream` and returns without
 * synchronising, so the caller may refill another chunk buffer meanwhile; an
 * index >= D is reported as FAST_EINVAL by the next call on the context that
 * synchronises (fast_build_tables on these keys does).
 */
fast_status fast_sig_rows(fast_ctx *ctx, const uint16_t *d_idx, uint64_t n, uint32_t ld, uint32_t *d_sig, uint64_t N,
                          uint64_t col0, void *stream);

/*
 * Hash-table construction (§6.1 "Hash table construction") and the
 * occurrence filter (§6.5).  Reads d_sig (b*N, table-major, as written by
 * fast_sig) and builds, per table, the (key, id) pairs stably sorted by key
 * -- each bucket a run of equal keys with ids ascending -- plus the drop mask.
 * N <= 2^28 - 1.  The tables live in device memory owned by *out.  d_sig
 * is not copied: it must stay valid and unchanged until fast_search on these
 * tables has returned (the search compares keys of fingerprint pairs).
 */
fast_status fast_build_tables(fast_ctx *ctx, const uint32_t *d_sig, uint64_t N, fast_tables **out,
                              void *stream);

/*
 * Device views of a table set: d_skey / d_sid are b*N uint32 (table t at
 * offset t*N), d_drop is N uint8 (1 = dropped by the occurrence filter).
 * Any out-pointer may be NULL.
 */
fast_status fast_tables_view(const fast_tables *tb, uint64_t *N, uint32_t *b, const uint32_t **d_skey,
                             const uint32_t **d_sid, const uint8_t **d_drop);

void fast_tables_free(fast_tables *tb);

/*
 * Search (§6.1 "Search", §6.3 detection threshold, §6.4 partitioned search,
 * §7.2 output triplets): every pair (i, j), i < j, neither dropped,
 * j - i > excl, sharing a bucket in votes >= v tables, sorted by (i, j).
 * `tb` must come from `ctx`.  Synchronises `stream`.
 */
fast_status fast_search(fast_ctx *ctx, const fast_tables *tb, fast_result **out, void *stream);

/*
 * The whole path, idx resident in HBM: fast_sig + fast_build_tables +
 * fast_search in one call, intermediates held in the context's workspace.
 */
fast_status fast_detect(fast_ctx *ctx, const uint16_t *d_idx, uint64_t N, uint32_t ld, fast_result **out,
                        void *stream);

/*
 * Batched search of several stations in one pass (pairs never cross
 * stations).  d_idx holds the stations' windows one after the other
 * (station x: h_station_N[x] rows of ld uint16, device memory); every stage
 * runs once over all of them -- one signature launch, one table sort with a
 * final stable pass on the station, one launch per search stage -- with each
 * station's own occurrence threshold (its own N).  out[x] receives station
 * x's detections with station-local ids, exactly those of fast_detect on that
 * station alone.  1 <= n_st <= 256; sum of the N < 2^28.
 */
fast_status fast_detect_batch(fast_ctx *ctx, const uint16_t *d_idx, const uint64_t *h_station_N, uint32_t n_st,
                              uint32_t ld, fast_result **out, void *stream);

/*
 * Batched search plans: a fixed batch shape whose table build (signatures,
 * radix passes, occurrence filter) is captured once as a CUDA graph and
 * replayed for every run, and whose search options are chosen by an
 * autotuner on the first run.  The plan reads d_idx, the device buffer given
 * at creation, on every run: refill that buffer between runs.  `stream` must
 * not be the legacy default stream (graph capture).  Creation runs the build
 * once (to size the plan's arena, which the plan then owns).
 */
typedef struct fast_plan fast_plan;

typedef struct {
    uint32_t vote_map;    /* 1 = global vote map, 0 = row-partitioned votes  */
    uint32_t large_min;   /* dense-group threshold (0 = automatic)           */
    float map_load;       /* vote-map load factor                            */
    float ms;             /* measured search time of this choice             */
    uint32_t group_pairs; /* pairs per row group of the row votes (0 = default) */
} fast_plan_choice;

typedef struct {
    uint64_t graph_nodes, graph_kernels, arena_bytes;
    float build_ms;      /* last replay of the build graph (timing option on) */
    uint32_t tuned, n_tried;
    fast_plan_choice best;
    fast_plan_choice tried[8];
} fast_plan_info_t;

fast_status fast_plan_create(fast_ctx *ctx, const uint16_t *d_idx, const uint64_t *h_station_N, uint32_t n_st,
                             uint32_t ld, void *stream, fast_plan **out);

/* Replays the build graph and searches; out[x] as fast_detect_batch gives.
 * The first run times every candidate option set (vote path, dense-group
 * threshold, row-group size, map load) and keeps the fastest for later runs; the context's
 * own options are left as they were.  Every candidate gives the same list. */
fast_status fast_plan_run(fast_plan *plan, fast_result **out, void *stream);

fast_status fast_plan_info(const fast_plan *plan, fast_plan_info_t *info);

void fast_plan_destroy(fast_plan *plan);

/*
 * The whole path from and to host memory: copies h_idx (N rows of ld uint16)
 * to the device, runs fast_detect, and copies at most `cap` detections back
 * to h_i / h_j / h_votes.  *M receives the total number of detections (which
 * may exceed cap; then only the first cap, in (i, j) order, are copied).
 */
fast_status fast_detect_host(fast_ctx *ctx, const uint16_t *h_idx, uint64_t N, uint32_t ld, uint64_t *M,
                             uint32_t *h_i, uint32_t *h_j, uint8_t *h_votes, uint64_t cap, void *stream);

/*
 * The whole path over a station whose fingerprints are produced in chunks by
 * the caller (§6.4 "Partition": a long station's data need not be held at
 * once): fill(user, row0, n, ld, h_rows) must write windows row0 .. row0+n-1
 * (n rows of ld uint16, ld >= K) into the pinned host buffer h_rows and
 * return 0 (non-zero aborts the call with FAST_EINVAL).  The library calls
 * it for consecutive chunks of chunk_rows windows (the last may be shorter),
 * on the calling thread, while the previous chunk is copied and signed on
 * the device: only two chunks of input are ever held, on the host and on the
 * device.  Then builds the tables (table_group at a time) and searches, as
 * fast_detect does; *out as fast_detect gives.  N < 2^28.  The staging
 * buffers (2 * chunk_rows * ld * 2 bytes of pinned host memory) are kept by
 * the context for later calls.  Synchronises `stream`.
 */
typedef int (*fast_fill_rows)(void *user, uint64_t row0, uint64_t n, uint32_t ld, uint16_t *h_rows);

fast_status fast_detect_chunked(fast_ctx *ctx, uint64_t N, uint32_t ld, uint64_t chunk_rows, fast_fill_rows fill,
                                void *user, fast_result **out, void *stream);

/*
 * Device views of a result: *M detections as three arrays (structure of
 * arrays), sorted by (i asc, j asc).  Any out-pointer may be NULL.
 */
fast_status fast_result_view(const fast_result *res, uint64_t *M, const uint32_t **d_i, const uint32_t **d_j,
                             const uint8_t **d_votes);

void fast_result_free(fast_result *res);

/* Stage times and counters of the last search on `ctx`. */
fast_status fast_get_stats(const fast_ctx *ctx, fast_stats *out);

/*
 * Tuning knobs; none changes any result.
 *   "large_min"  live bucket size from which buckets are summed by direct key
 *                comparison inside groups instead of the vote map (0 = auto)
 *   "map_load"   target load factor of the vote map, in (0.05, 0.95)
 *   "group_pairs" expected sparse pairs per row group of the row-partitioned
 *                vote, 0 (= 1024) or in [64, 8192]
 *   "timing"     1 = record per-stage CUDA events (default), 0 = off
 *   "vote_map"   1 = sum sparse votes in one global open-addressing map of
 *                packed (i, j) -> votes and order the list by a radix sort;
 *                0 = count them row by row (default)
 *   "single_pass" 1 = write the row groups' pairs in one pass over the tables
 *                into fixed-size group regions (with an overflow list), then
 *                compact them, when one row partition is used and the regions
 *                fit the budget (default); 0 = count the pairs in a first
 *                pass and write them at exact offsets in a second
 *   "group_slots" region slots per row group of the single pass, 0 (= about
 *                twice the expected pairs per group) or in [1, 65536]; pairs
 *                past them go through the overflow list
 *   "dense_masks" 1 = vote dense groups from cluster bit masks when their
 *                scratch fits the memory (default), 0 = always by direct
 *                comparison of the members' keys (what the search falls back
 *                to when the masks' scratch does not fit)
 */
fast_status fast_set_option(fast_ctx *ctx, const char *name, double value);

/* ------------------------------------------------------------------ */
/* Streaming search server                                             */
/* ------------------------------------------------------------------ */
/*
 * A server keeps, per station, the hash tables of a preloaded history
 * resident in HBM and answers requests -- batches of new windows of one
 * station -- against the history and every earlier batch of that station
 * (the tables stay populated while new fingerprints query them, §6.4
 * "Partition"; each new fingerprint queries its buckets, §6.1 "Search").
 *
 * Semantics.  Window ids continue the station timeline: the history is
 * 0..N0-1, each submitted batch takes the next n ids in submission order.
 * Request q reports every pair (i, j) with j in its batch and i < j (i in the
 * history, an earlier batch of the station, or its own batch), neither
 * dropped, j - i > excl, votes >= v, sorted by (i, j).  History windows keep
 * the drop flag of the history alone (occurrence filter on the N0 windows);
 * a later window is dropped iff its key falls in a heavy history bucket
 * (occ_den * size > occ_num * N0) in more than b/2 tables.  The result of a
 * request depends only on the station's submission sequence, never on the
 * timing or interleaving of other requests.
 *
 * Execution.  One worker thread and one CUDA stream per station: a station's
 * requests run in submission order, different stations run concurrently on
 * the device.  A request starts when an estimate of its working set fits the
 * HBM budget next to the requests already running (continuous admission as
 * memory frees up).  Thread safety: submit / poll / latency / release may be
 * called from any host thread.
 */
typedef struct fast_server fast_server;

/*
 * Creates a server with n_stations stations (1..1024) on the current
 * device.  max_stream_windows bounds the windows each station may receive
 * after its history (the device delta tables are sized for it);
 * hbm_budget_bytes bounds resident tables plus running requests (0 = none).
 */
fast_status fast_server_create(const fast_params *p, uint32_t n_stations, uint64_t max_stream_windows,
                               uint64_t hbm_budget_bytes, fast_server **out);

/* Stops the workers (queued requests fail with FAST_ETIMEOUT) and frees all. */
void fast_server_destroy(fast_server *srv);

const char *fast_server_last_error(const fast_server *srv);

/*
 * Loads a station's history (N rows of ld uint16 indices, host memory):
 * signs it, builds and keeps its tables, applies the occurrence filter.
 * Synchronous.  Must precede the station's first submit; at most once.
 */
fast_status fast_server_load_history(fast_server *srv, uint32_t station, const uint16_t *h_idx, uint64_t N,
                                     uint32_t ld);

/*
 * Queues a batch of n >= 1 new windows (host memory, n rows of ld uint16)
 * for `station` and returns its request id.  The input is copied before the
 * call returns.
 */
fast_status fast_stream_submit(fast_server *srv, uint32_t station, const uint16_t *h_idx, uint32_t n, uint32_t ld,
                               uint64_t *req_id);

/*
 * Waits up to timeout_us microseconds for a request.  FAST_EPENDING if it is
 * not finished; the request's own error if it failed; FAST_OK with its
 * detections otherwise: *M pairs as host arrays (valid until
 * fast_stream_release) and *first_id, the id of the batch's first window.
 */
fast_status fast_stream_poll(fast_server *srv, uint64_t req_id, uint64_t timeout_us, uint64_t *M, uint64_t *first_id,
                             const uint32_t **h_i, const uint32_t **h_j, const uint8_t **h_votes);

/* Seconds from submit to completion of a finished request. */
fast_status fast_stream_latency(fast_server *srv, uint64_t req_id, double *seconds);

/* Forgets a finished request and frees its results. */
fast_status fast_stream_release(fast_server *srv, uint64_t req_id);

/*
 * fast_set_option on every station's context; before any history is loaded.
 * One server setting is also taken here, at any time:
 *   "admit_timeout_ms"  the longest a request waits for admission (its
 *                       working set to fit the HBM budget next to the running
 *                       requests), in [0, 86400000] ms, default 300000; a
 *                       request still waiting then fails with FAST_ETIMEOUT.
 */
fast_status fast_server_set_option(fast_server *srv, const char *name, double value);

/*
 * Test hook: reserves `bytes` of the admission budget as if a request that
 * never finishes were running (0 gives it back).  Requests that no longer fit
 * wait for admission, and fail with FAST_ETIMEOUT once admit_timeout_ms ends.
 */
fast_status fast_server_hold_budget(fast_server *srv, uint64_t bytes);

/*
 * Test hook: the request with id req_id fails on the host (FAST_EINTERNAL)
 * instead of running; every other request is unaffected.
 */
fast_status fast_server_inject_failure(fast_server *srv, uint64_t req_id);

/*
 * Query-only hashing (§6.4 "Partition", last paragraph: hash only the query
 * items, then check every other item against their buckets).  d_batch holds
 * n new windows (ld >= K uint16 each) that follow a station's N0 history
 * windows d_hist on its timeline (ids N0 .. N0 + n - 1).  Only the batch is
 * put into hash tables; the history's keys are computed and streamed past
 * them, so no table of the history is built.  *out receives every pair
 * (i, j) with j in the batch and i < j (i in the history or the batch),
 * neither dropped, j - i > excl, votes >= v, sorted by (i, j) -- the same
 * list as the batch streamed to a server right after that history
 * (fast_stream_submit).  d_hist_drop: N0 flags (1 = dropped) of the history
 * windows, e.g. fast_tables_view's drop mask of the history; NULL = none
 * dropped.  A batch window is dropped when its key falls in a heavy history
 * bucket (occ_den * size > occ_num * N0, sizes over all N0 history windows)
 * in more than b/2 tables.  N0 + n < 2^28.  Synchronises `stream`.
 */
fast_status fast_query_only(fast_ctx *ctx, const uint16_t *d_hist, uint64_t N0, const uint8_t *d_hist_drop,
                            const uint16_t *d_batch, uint64_t n, uint32_t ld, fast_result **out, void *stream);

/* ------------------------------------------------------------------ */
/* Alignment: the steps that take the search's output (§7)             */
/* ------------------------------------------------------------------ */
typedef struct fast_merged fast_merged;
typedef struct fast_clusters fast_clusters;

/*
 * Channel level (§7.1 "Channel Level"; §7.2, the sort-merge-reduce
 * procedure): the similarity lists of nch channels of one station are summed
 * per pair and the pairs whose summed votes reach thr are kept ("a slightly
 * higher similarity threshold on the combined similarity matrix").
 *   N          windows of the station: every id of every list is < N;
 *              2 <= N <= 2^28.
 *   nch        channels, 1..256; channel c has h_M[c] entries d_i[c][k],
 *              d_j[c][k], d_votes[c][k] (device arrays; h_M, d_i, d_j,
 *              d_votes are host arrays of nch entries), each with i < j and
 *              each pair at most once per channel (a fast_search result
 *              qualifies, in any order).
 * *out receives the kept pairs (i, j, sim), sim the summed votes (16 bits),
 * in the paper's merged order: dt = j - i ascending, then idx1 = i
 * ascending.  An entry with j <= i or j >= N makes the call fail with
 * FAST_EINVAL.  Synchronises `stream`.  The inputs are not modified.
 */
fast_status fast_channel_merge(fast_ctx *ctx, uint64_t N, uint32_t nch, const uint64_t *h_M,
                               const uint32_t *const *d_i, const uint32_t *const *d_j,
                               const uint8_t *const *d_votes, uint32_t thr, fast_merged **out, void *stream);

/* Device views of a merged list: *M entries as three arrays.  Any out-pointer may be NULL. */
fast_status fast_merged_view(const fast_merged *res, uint64_t *M, const uint32_t **d_i, const uint32_t **d_j,
                             const uint16_t **d_sim);

void fast_merged_free(fast_merged *res);

/*
 * Station level (§7.1 "Station Level"; §7.2 "Station"): thin diagonal
 * clusters of a station's combined similarity list, each reduced to summary
 * statistics, small ones pruned.
 *   Input: n entries (d_i, d_j, d_sim; device arrays) in strictly increasing
 *   (dt = j - i, idx1 = i) order, as fast_channel_merge returns them;
 *   n < 2^32 - 1.  Otherwise the call fails with FAST_EINVAL.
 *   runs     along every diagonal dt, the maximal sequences of entries whose
 *            consecutive idx1 differ by less than `gap` (gap >= 1);
 *   merge    each run, in (dt, idx1) order, joins the first cluster on
 *            diagonal dt - 1 it comes within `gap` of (idx1 ranges
 *            [s, e] and [s', e'] are near when s <= e' + gap - 1 and
 *            s' <= e + gap - 1) if the joined cluster then spans at most
 *            `width` diagonals (width >= 1), else it starts its own;
 *   summary  per cluster: dt_min, dt_max, idx1_min, idx1_max (idx1 of the
 *            first and last entry of its runs), entries, summed sim;
 *   prune    clusters of fewer than min_n entries are dropped.
 * *out receives 6 uint64 per cluster in that order, clusters in
 * (dt_min, idx1_min) order (ties in the order of their first runs).
 * Synchronises `stream`.
 */
fast_status fast_station_clusters(fast_ctx *ctx, const uint32_t *d_i, const uint32_t *d_j, const uint16_t *d_sim,
                                  uint64_t n, uint32_t gap, uint32_t width, uint32_t min_n, fast_clusters **out,
                                  void *stream);

/* Device view of the clusters: *n rows of 6 uint64. */
fast_status fast_clusters_view(const fast_clusters *res, uint64_t *n, const uint64_t **d_box);

void fast_clusters_free(fast_clusters *res);

/*
 * One table's stable (key, id) sort without any device allocation.
 * No counterpart in the paper: this is a service entry point of this library.
 *
 * Some callers cannot let a library call cudaMalloc: hosts that plan all
 * device memory themselves up front (a serving process that has already
 * reserved the GPU's memory for its own pools, so any further driver
 * allocation fails or would break its budget), and latency-bound callers for
 * which cudaMalloc's implicit device-wide synchronisation is unacceptable.
 * This entry point sorts d_keys[0..n) by key, stably, and writes d_skey[k] /
 * d_sid[k] = the k-th (key, original index) pair: the same listing as one
 * table of fast_build_tables.
 *
 * The caller passes the input and both outputs (n uint32 each, device
 * memory, not overlapping).  The scratch (one ping-pong pair of keys and ids
 * plus digit counts, about 8.9 MB) is a fixed array inside the library: every
 * GPU that loads the library holds it until the process exits.
 *   - n <= 1048576 (2^20); larger n returns FAST_EINVAL and does nothing.
 *   - The first call on a device looks up the array's device address (once
 *     per device, on the current device); make that first call before any
 *     stream capture.
 *   - All calls on a device share the array: calls whose GPU work overlaps
 *     (different streams, or host threads without ordering) race and corrupt
 *     each other's results.  Order them on one stream or synchronise between
 *     them.  Every scratch word a call reads is written earlier in the same
 *     call, so nothing left by a previous call leaks into the result.
 * Returns FAST_OK once the work is enqueued on `stream`, FAST_EINVAL for bad
 * arguments, FAST_ECUDA if a CUDA call fails -- also, before anything is
 * launched, when an error of earlier work is pending on the calling thread
 * (that error is left in place for the caller to read).
 */
fast_status fast_table_sort_static(const uint32_t *d_keys, uint64_t n, uint32_t *d_skey, uint32_t *d_sid,
                                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FAST_H */
