// fast_internal.cuh -- shared definitions of the GB300 search library.
//
// Device side: SplitMix64 mixing used by the hash parameters and by
// hash_combine (Algorithm 1), device error flags, launch helpers.
// Host side: the context (parameters, per-function rank tables, memory pool,
// stage timers) and the stream-ordered allocator with the HBM budget.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fast.h"

namespace fastgb {

// ----------------------------------------------------------------- device

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// SplitMix64 finaliser (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// n-th SplitMix64 output for `seed`.
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t n) {
    return mix64(seed + (n + 1) * kGamma);
}

// h(x) = high 32 bits of a*x + b (mod 2^64): one 32x32->64 multiply-add of
// the low half of a plus a 32-bit multiply-add of the high half.
__device__ __forceinline__ uint32_t hash_ab(uint32_t a_lo, uint32_t a_hi, uint64_t b, uint32_t x) {
    uint64_t t = (uint64_t)a_lo * x + b;
    return (uint32_t)(t >> 32) + a_hi * x;
}

// A batched search concatenates stations: station s holds window ids and
// table positions [soff[s], soff[s+1]) (soff has nst + 1 entries; a single
// station is nst = 1, soff = {0, N}).  Buckets never cross a station.
struct Stations {
    const uint64_t *soff;
    uint32_t nst;
};

__device__ __forceinline__ uint32_t station_of(const Stations &S, uint64_t p) {
    uint32_t lo = 0, hi = S.nst;  // largest s with soff[s] <= p
    while (hi - lo > 1) {
        const uint32_t m = (lo + hi) / 2;
        if (S.soff[m] <= p) lo = m;
        else hi = m;
    }
    return lo;
}

// Device error flags, OR-ed into ctx->d_err.
enum : uint32_t {
    ERR_BAD_INDEX = 1u << 0,   // fingerprint index >= D
    ERR_MAP_FULL = 1u << 1,    // vote map probe limit
    ERR_OVERFLOW = 1u << 2,    // an output / list capacity was exceeded
    ERR_WALK = 1u << 3,        // signature walk ran off the end (bad input)
    ERR_INTERNAL = 1u << 4,
    ERR_INPUT = 1u << 5,       // an input list breaks its stated order or range
};

__device__ __forceinline__ void set_err(uint32_t *err, uint32_t bit) { atomicOr(err, bit); }

// Device open-addressing vote map: one 64-bit slot per pair, i:28 | j:28 |
// votes:8 (0 = empty), capacity `cap` slots, linear probing.
struct Map {
    unsigned long long *slot;
    uint64_t cap;
};

__device__ __forceinline__ uint64_t pair_key(uint32_t i, uint32_t j) { return ((uint64_t)i << 28) | j; }

// Adds one vote to (i, j).  Slot = key56 << 8 | votes; 0 = empty.
__device__ __forceinline__ void map_add(Map m, uint64_t key56, uint32_t *err) {
    const unsigned long long want = (unsigned long long)(key56 << 8);
    uint64_t h = __umul64hi(mix64(key56), m.cap);
    for (uint32_t probe = 0; probe < 1u << 16; probe++) {
        unsigned long long cur = __ldcg(m.slot + h);
        if (cur == 0) {
            unsigned long long old = atomicCAS(m.slot + h, 0ull, want | 1ull);
            if (old == 0) return;
            cur = old;
        }
        if ((cur & ~0xFFull) == want) {
            atomicAdd(m.slot + h, 1ull);
            return;
        }
        if (++h == m.cap) h = 0;
    }
    set_err(err, ERR_MAP_FULL);
}

// Adds `n` votes to (i, j) (n <= 255 - current votes, always true: votes <= b).
__device__ __forceinline__ void map_add_n(Map m, uint64_t key56, uint32_t n, uint32_t *err) {
    const unsigned long long want = (unsigned long long)(key56 << 8);
    uint64_t h = __umul64hi(mix64(key56), m.cap);
    for (uint32_t probe = 0; probe < 1u << 16; probe++) {
        unsigned long long cur = __ldcg(m.slot + h);
        if (cur == 0) {
            unsigned long long old = atomicCAS(m.slot + h, 0ull, want | n);
            if (old == 0) return;
            cur = old;
        }
        if ((cur & ~0xFFull) == want) {
            atomicAdd(m.slot + h, (unsigned long long)n);
            return;
        }
        if (++h == m.cap) h = 0;
    }
    set_err(err, ERR_MAP_FULL);
}


// ------------------------------------------------------------------- host

struct StageTimer;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace fastgb

constexpr int kCopyChunks = 8;

struct fast_ctx {
    fast_params p{};
    int device = 0;
    int num_sms = 0;
    uint32_t F = 0;        // hash functions
    uint32_t W = 0;        // walks: F (MinHash) or 2F (Min-Max)
    bool use_walk = false;
    uint32_t Dpad = 0;     // walk sequence length (multiple of 8)
    // device constants
    uint64_t *d_a = nullptr;      // [F]
    uint64_t *d_b = nullptr;      // [F]
    uint64_t *d_zinit = nullptr;  // [b] combine start values
    uint16_t *d_walk = nullptr;   // [W][Dpad] x in ascending (min walks) / descending (max walks) h order
    uint32_t *d_err = nullptr;    // device error flags
    uint64_t *d_scal = nullptr;   // small device scalars (counters), kScal entries
    uint64_t *h_scal = nullptr;   // pinned mirror
    // memory
    cudaMemPool_t pool = nullptr;
    uint64_t budget = 0;   // 0 = unbounded
    uint64_t live = 0;     // bytes currently allocated through the pool
    uint64_t peak = 0;
    // arena mode (CUDA-graph capture): allocations bump-allocate from a fixed
    // buffer and frees are no-ops; trace mode sums the bytes allocated
    char *arena = nullptr;
    uint64_t arena_size = 0, arena_off = 0;
    bool trace = false;
    uint64_t trace_total = 0;
    bool capturing = false;     // no host synchronisation while a graph is being captured
    // tuning
    uint32_t large_min = 0;     // live bucket size from which a bucket goes to the dense path (0 = auto)
    uint32_t group_pairs = 0;   // expected sparse pairs per row group of the vote (0 = 1024)
    float map_load = 0.5f;      // vote-map load factor target
    bool vote_map = false;      // sum sparse votes in one global hash map instead of per row
    bool single_pass = true;    // write the sparse pairs in one pass (fixed group regions) when they fit
    uint32_t group_slots = 0;   // region slots per row group of the single pass (0 = about twice the expected)
    bool dense_masks = true;    // vote dense groups from cluster masks when their scratch fits
    // instrumentation
    fast_stats stats{};
    cudaEvent_t ev[24] = {};
    // host entry: input copied in chunks on a second stream while the signature kernel runs
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t cev[kCopyChunks + 1] = {};
    // chunked host input (fast_detect_chunked): two pinned staging buffers,
    // their copy-done and consumed events
    uint16_t *h_stage[2] = {};
    size_t h_stage_bytes = 0;
    cudaEvent_t chev[4] = {};
    bool timing = true;
    int last_stage = 0;  // the most recent stage mark (named in allocation failures)
    // the key array of the current call when the library allocated it: the
    // search gives it back as soon as the dense groups have their keys
    uint32_t *sig_owned = nullptr;
    size_t sig_owned_bytes = 0;
    std::string err;
};

struct fast_tables {
    fast_ctx *ctx = nullptr;
    uint64_t N = 0;
    uint32_t b = 0;
    const uint32_t *d_sig = nullptr;  // [b][N] keys the tables were built from (caller-owned)
    uint32_t nst = 1;                 // stations (batched search)
    std::vector<uint64_t> soff;       // [nst + 1] station offsets (host)
    uint64_t *d_soff = nullptr;       // same, device
    uint32_t *d_skey = nullptr;  // [b][N]
    uint32_t *d_sid = nullptr;   // [b][N]
    uint8_t *d_drop = nullptr;   // [N]
    uint64_t n_dropped = 0;
    // buckets of more than 32 entries (table, start, end, 0), found once by
    // the filter and reused by the search; d_bigcnt = {count, small-bucket pairs}
    uint4 *d_big = nullptr;
    uint64_t big_cap = 0;
    unsigned long long *d_bigcnt = nullptr;
    cudaStream_t stream = nullptr;
};

struct fast_result {
    fast_ctx *ctx = nullptr;
    uint64_t M = 0;
    uint32_t *d_i = nullptr;
    uint32_t *d_j = nullptr;
    uint8_t *d_votes = nullptr;
    cudaStream_t stream = nullptr;
};

#define FAST_LAUNCHED(c) ((c)->stats.n_launches++)

namespace fastgb {

constexpr int kScal = 128;

// Stream-ordered allocation from the context's pool, checked against the budget.
fast_status dalloc(fast_ctx *c, void **p, size_t bytes, cudaStream_t s);
void dfree(fast_ctx *c, void *p, size_t bytes, cudaStream_t s);

template <typename T>
inline fast_status dalloc_t(fast_ctx *c, T **p, size_t count, cudaStream_t s) {
    return dalloc(c, reinterpret_cast<void **>(p), count * sizeof(T), s);
}

fast_status set_error(fast_ctx *c, fast_status st, const std::string &msg);
fast_status cuda_fail(fast_ctx *c, cudaError_t e, const char *where);

// Synchronises `s` and converts device error flags into a status.
fast_status sync_check(fast_ctx *c, cudaStream_t s, const char *where);

inline unsigned ceil_div(uint64_t a, uint64_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ kernel launchers
// k_sig.cu
fast_status sig_setup(fast_ctx *c);
fast_status sig_launch(fast_ctx *c, const uint16_t *d_idx, uint64_t N, uint32_t ld, uint32_t *d_sig,
                       cudaStream_t s);
// N rows of d_idx whose keys go to columns [0, N) of a [b][Nst] key array
// (d_sig already offset to the first column): one chunk of a larger batch.
fast_status sig_launch_rows(fast_ctx *c, const uint16_t *d_idx, uint64_t N, uint32_t ld, uint32_t *d_sig, uint64_t Nst,
                            cudaStream_t s);

// k_sort.cu: stable LSD radix sort of `nseg` equal segments of length `len`.
// Keys in/out, optional 32-bit values (vals_in == nullptr -> values are the
// element index within its segment).  Sorts on bits [bit0, bit1).  Result is
// left in (keys_out, vals_out); keys_tmp/vals_tmp are scratch of equal size.
struct SortScratch {
    uint32_t *counts = nullptr;   // [nseg][256][nchunks]
    uint64_t *offsets = nullptr;  // [nseg][256][nchunks]
    size_t cap_entries = 0;
};
// With stations (S.nst > 1, device offsets), each of the nseg rows is sorted
// station by station (seg_max: the longest station), which orders it by
// (station, key, id).
fast_status sort_u32(fast_ctx *c, uint32_t nseg, uint64_t len, const uint32_t *keys_in, const uint32_t *vals_in,
                     uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, uint32_t bit0,
                     uint32_t bit1, uint32_t **keys_out, uint32_t **vals_out, cudaStream_t s, uint32_t *passes,
                     Stations S = Stations{nullptr, 1}, uint64_t seg_max = 0);
fast_status sort_u64(fast_ctx *c, uint64_t len, uint64_t *keys_a, uint64_t *keys_b, uint32_t bit0, uint32_t bit1,
                     uint64_t **keys_out, cudaStream_t s);

// k_scan.cu: out[seg][k] = sum of in[seg][0..k), nseg segments of n counts;
// totals[seg] (optional, device) receives each segment's sum.
fast_status scan_excl(fast_ctx *c, const uint32_t *in, uint64_t *out, uint64_t n, uint32_t nseg, uint64_t *totals,
                      cudaStream_t s);

// k_search.cu
fast_status filter_launch(fast_ctx *c, fast_tables *tb, cudaStream_t s);
fast_status search_run(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, fast_result **out,
                       cudaStream_t s);

// Dense groups of a station's history, kept resident by the streaming server:
// components of large buckets (live size >= large_min), their members, the
// members' keys, and every table's large buckets with their group.
struct HistGroups {
    uint32_t large_min = 0;
    uint64_t nm = 0, ng = 0, nlarge = 0;
    uint32_t *label = nullptr;   // [N0] group index of each window, ~0 outside groups
    uint32_t *ids = nullptr;     // [nm] members, sorted by (group, id)
    uint32_t *GT = nullptr;      // [b][nm] members' keys
    uint32_t *gstart = nullptr;  // [ng + 1] member offsets of each group
    uint4 *large = nullptr;      // [nlarge] (table, start, end, group), sorted by (table, start)
    uint32_t *tstart = nullptr;  // [b + 1] first large bucket of each table in `large`
    uint32_t *bm = nullptr;      // membership bitmaps: bit m of large bucket x = member m of its group
    uint64_t *bm_off = nullptr;  // [nlarge] first word of each large bucket's bitmap
};
fast_status history_groups(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, HistGroups *g, cudaStream_t s);
uint32_t large_min_for(const fast_ctx *c, uint64_t N);  // the dense-group threshold (option or automatic)
uint64_t room_bytes(const fast_ctx *c);                 // device memory a call may still take
void sig_release(fast_ctx *c, cudaStream_t s);          // frees the call's own key array, if any
struct Scal {  // device scalar slots (ctx->d_scal)
    enum { NBIG, NLARGE, NMEDIUM, NHEAVY, NDROP, NMEMB, CUR_DENSE, CUR_SPARSE, CHANGED, NLONG, NMERGE, NMERGE_TOT,
           NCAND, NMID, SMALLPAIRS, NSMALLEMIT, NSLOW, NOVF, LMAX, NMEDW, NMEDF, NMEDB, NMEDH, MEDNEXT, MEDNEXTH,
           PART0 };
};
void history_groups_free(HistGroups *g);

// fast_api.cu
fast_status split_stations(fast_ctx *c, fast_result *all, const std::vector<uint64_t> &soff, fast_result **out,
                           cudaStream_t s);
}  // namespace fastgb
fast_status build_tables(fast_ctx *c, const uint32_t *d_sig, uint64_t N, const uint64_t *h_soff, uint32_t nst,
                         fast_tables **out, cudaStream_t s);
void stats_times(fast_ctx *c, bool whole);
namespace fastgb {
void stage_reset();  // forget the stage marks of the previous call on this thread

// timing helpers (fast_api.cu)
void stage_mark(fast_ctx *c, int slot, cudaStream_t s);
float stage_ms(fast_ctx *c, int a, int b);

}  // namespace fastgb
