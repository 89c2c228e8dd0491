// serve.cu -- streaming search server (serving form of §6.4 "Partition":
// the hash tables stay populated while new fingerprints are queried
// against them, and §6.1 "Search": each new fingerprint queries its buckets).
//
// Per station the device holds the preloaded history as sorted tables (key,
// id) with its drop mask, plus a "delta": every later window already
// admitted, in a per-table multimap key -> ids (open-addressing slots of
// key:32 | head+1:32, entries chained by `next`).  A request (a batch of n new
// windows of one station, ids continuing the station timeline) is processed
// by its station's worker thread on the station's stream:
//   sign the batch -> look every (table, window) key up in the history
//   (binary search) -> frozen occurrence filter for the new windows -> sort
//   the batch's keys per table -> count candidates (history bucket + delta
//   chain + earlier same-key windows of the batch) -> add every candidate
//   pair to a request vote map -> keep votes >= v -> canonical (i, j) order ->
//   host -> insert the batch's live windows into the delta.
// Requests of one station run in admission order, so request q sees history,
// every earlier batch of its station and itself; stations run concurrently,
// each on its own stream, as HBM budget admits them.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "fast_internal.cuh"

namespace fastgb {
namespace {

constexpr uint32_t kNoneId = 0xFFFFFFFFu;

// Lower / upper bound of `key` in a sorted array.
__device__ __forceinline__ void equal_range(const uint32_t *k, uint64_t n, uint32_t key, uint64_t *lo_out,
                                            uint64_t *hi_out) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t m = (lo + hi) / 2;
        if (k[m] < key) lo = m + 1;
        else hi = m;
    }
    uint64_t a = lo;
    hi = n;
    while (lo < hi) {
        uint64_t m = (lo + hi) / 2;
        if (k[m] <= key) lo = m + 1;
        else hi = m;
    }
    *lo_out = a;
    *hi_out = lo;
}

__device__ __forceinline__ uint64_t dslot_hash(uint32_t key, uint64_t cap) {
    return __umul64hi(mix64((uint64_t)key * 0x9E3779B97F4A7C15ull + 1), cap);
}

// Head (entry index + 1, 0 = none) of the delta chain of `key`.
__device__ __forceinline__ uint32_t delta_head(const unsigned long long *slot, uint64_t cap, uint32_t key) {
    if (cap == 0) return 0;
    uint64_t h = dslot_hash(key, cap);
    for (uint64_t probe = 0; probe < cap; probe++) {
        const unsigned long long cur = slot[h];
        if (cur == 0) return 0;
        if ((uint32_t)(cur >> 32) == key) return (uint32_t)cur;
        if (++h == cap) h = 0;
    }
    return 0;
}

struct ReqArgs {
    // history
    const uint32_t *hkey, *hid;
    const uint8_t *hdrop;
    uint64_t N0;
    // delta
    const unsigned long long *dslot;
    const uint32_t *dent_id, *dent_next;
    uint64_t dcap_k, dcap_e;
    // batch
    const uint32_t *keys;   // [b][n] batch keys
    const uint32_t *bkey;   // [b][n] batch keys sorted per table
    const uint32_t *bid;    // [b][n] local window of each sorted entry
    const uint32_t *bpos;   // [b][n] sorted position of local window w
    const uint2 *range;     // [b][n] history bucket [lo, hi) of each (table, window)
    const uint8_t *ndrop;   // [n] dropped new windows
    uint32_t n, nb, excl;
    uint64_t first_id;
    uint32_t occ_num, occ_den;
    // dense groups of the history
    const uint32_t *label;   // [N0] group index of each history window (~0 = none)
    const uint4 *large;      // large buckets (table, start, end, group), by (table, start)
    const uint32_t *tstart;  // [b + 1]
    uint32_t *wg;            // [n][kWG] groups a window meets in large buckets (~0 = free)
};

constexpr uint32_t kWG = 4;            // groups tracked per new window
constexpr uint32_t kLargeFlag = 0x80000000u;

// History bucket of every (table, window); heavy-bucket counts for the frozen
// filter; a bucket listed as large is flagged and its group recorded for the
// window (when the window already tracks kWG other groups the bucket stays
// in the sparse path -- any split is exact as long as a group is wholly
// dense or wholly sparse for the window).
__global__ void k_req_lookup(ReqArgs a, uint2 *__restrict__ range, uint32_t *__restrict__ hcnt) {
    const uint32_t t = blockIdx.y;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.n; w += gridDim.x * blockDim.x) {
        uint64_t lo, hi;
        equal_range(a.hkey + (uint64_t)t * a.N0, a.N0, a.keys[(uint64_t)t * a.n + w], &lo, &hi);
        uint32_t flag = 0, x_large = 0;
        if (hi > lo) {
            uint32_t x0 = a.tstart[t], x1 = a.tstart[t + 1];  // large buckets of table t, by start
            while (x0 < x1) {
                const uint32_t m = (x0 + x1) / 2;
                if (a.large[m].y < lo) x0 = m + 1;
                else x1 = m;
            }
            if (x0 < a.tstart[t + 1] && a.large[x0].y == lo) {
                const uint32_t g = a.large[x0].w;
                uint32_t *slot = a.wg + (uint64_t)w * kWG;
                for (uint32_t k = 0; k < kWG; k++) {
                    const uint32_t old = atomicCAS(slot + k, kNoneId, g);
                    if (old == kNoneId || old == g) {
                        flag = kLargeFlag;
                        x_large = x0;
                        break;
                    }
                }
            }
        }
        // a flagged range carries the large bucket's index instead of its start
        range[(uint64_t)t * a.n + w] = make_uint2(flag ? x_large : (uint32_t)lo, (uint32_t)hi | flag);
        if (a.occ_num && (uint64_t)a.occ_den * (hi - lo) > (uint64_t)a.occ_num * a.N0) atomicAdd(hcnt + w, 1u);
    }
}

// Dense part of a request: for each group window w meets in large history
// buckets, the votes of every member i from those buckets are the number of
// the buckets' membership bitmaps holding i; they enter the request's vote map
// as one addition per member.  One CTA per window.
template <int MODE>
__global__ void k_req_dense(ReqArgs a, const uint32_t *__restrict__ gstart, const uint32_t *__restrict__ ids,
                            const uint32_t *__restrict__ bm, const uint64_t *__restrict__ bm_off,
                            unsigned long long *__restrict__ total, unsigned long long *__restrict__ map,
                            uint64_t map_cap, uint32_t *err) {
    extern __shared__ uint32_t s_bk[];  // [nb] large-bucket index per table of this window's group, ~0 = none
    const uint32_t w = blockIdx.x;
    if (w >= a.n || a.ndrop[w]) return;  // block-uniform
    const uint64_t j = a.first_id + w;
    unsigned long long mine = 0;
    for (uint32_t k = 0; k < kWG; k++) {
        const uint32_t g = a.wg[(uint64_t)w * kWG + k];
        if (g == kNoneId) break;  // slots fill in order
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < a.nb; t += blockDim.x) {
            const uint2 rg = a.range[(uint64_t)t * a.n + w];
            s_bk[t] = ((rg.y & kLargeFlag) && a.large[rg.x].w == g) ? rg.x : kNoneId;
        }
        __syncthreads();
        const uint32_t g0 = gstart[g], gn = gstart[g + 1] - g0;
        if (MODE == 0) {
            if (threadIdx.x == 0) mine += gn;
            continue;
        }
        for (uint32_t x = threadIdx.x; x < (gn + 31) / 32; x += blockDim.x) {
            uint32_t cnt[32];
#pragma unroll
            for (int q = 0; q < 32; q++) cnt[q] = 0;
            for (uint32_t t = 0; t < a.nb; t++) {
                const uint32_t bx = s_bk[t];
                if (bx == kNoneId) continue;
                const uint32_t word = bm[bm_off[bx] + x];
#pragma unroll
                for (int q = 0; q < 32; q++) cnt[q] += (word >> q) & 1u;
            }
#pragma unroll
            for (int q = 0; q < 32; q++) {
                if (!cnt[q]) continue;
                const uint32_t m = x * 32 + q;
                const uint32_t i = ids[g0 + m];
                if (j - i > a.excl) {
                    Map mp{map, map_cap};
                    map_add_n(mp, pair_key(i, (uint32_t)j), cnt[q], err);
                }
            }
        }
    }
    if (MODE == 0 && threadIdx.x == 0 && mine) atomicAdd(total, mine);
}

__global__ void k_req_drop(const uint32_t *__restrict__ hcnt, uint32_t n, uint32_t nb, uint8_t *__restrict__ ndrop) {
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < n; w += gridDim.x * blockDim.x)
        ndrop[w] = (uint8_t)(2ull * hcnt[w] > nb);
}

__global__ void k_req_inverse(const uint32_t *__restrict__ bid, uint32_t n, uint32_t *__restrict__ bpos) {
    const uint32_t t = blockIdx.y;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        bpos[(uint64_t)t * n + bid[(uint64_t)t * n + x]] = x;
}

// Candidates of new window w in table t: history bucket members, delta chain
// members with the same key, earlier windows of the batch with the same key.
// MODE 0 counts them (an upper bound on the pairs), MODE 1 votes.
template <int MODE>
__global__ void k_req_pairs(ReqArgs a, unsigned long long *__restrict__ total, unsigned long long *__restrict__ map,
                            uint64_t map_cap, uint32_t *err) {
    const uint32_t t = blockIdx.y;
    unsigned long long mine = 0;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.n; w += gridDim.x * blockDim.x) {
        if (a.ndrop[w]) continue;
        const uint64_t j = a.first_id + w;
        const uint64_t tw = (uint64_t)t * a.n + w;
        const uint32_t key = a.keys[tw];
        const uint2 rg = a.range[tw];
        const uint32_t *hid = a.hid + (uint64_t)t * a.N0;
        // history members (i < N0 <= j); large buckets come from the bitmaps
        if (!(rg.y & kLargeFlag)) {
            if (MODE == 0) {
                mine += rg.y - rg.x;
            } else {
                for (uint32_t q = rg.x; q < rg.y; q++) {
                    const uint32_t i = hid[q];
                    if (!a.hdrop[i] && j - i > a.excl) {
                        Map m{map, map_cap};
                        map_add(m, pair_key(i, (uint32_t)j), err);
                    }
                }
            }
        }
        // earlier batches (delta): every entry is live and older than j
        const unsigned long long *slot = a.dslot + (uint64_t)t * a.dcap_k;
        const uint32_t *did = a.dent_id + (uint64_t)t * a.dcap_e;
        const uint32_t *dnx = a.dent_next + (uint64_t)t * a.dcap_e;
        for (uint32_t x = delta_head(slot, a.dcap_k, key); x; x = dnx[x - 1]) {
            const uint32_t i = did[x - 1];
            if (MODE == 0) {
                ++mine;
            } else if (j - i > a.excl) {
                Map m{map, map_cap};
                map_add(m, pair_key(i, (uint32_t)j), err);
            }
        }
        // earlier windows of this batch: the run before w's sorted position
        const uint32_t *bk = a.bkey + (uint64_t)t * a.n;
        const uint32_t *bi = a.bid + (uint64_t)t * a.n;
        for (int64_t y = (int64_t)a.bpos[tw] - 1; y >= 0 && bk[y] == key; y--) {
            const uint32_t w2 = bi[y];
            if (MODE == 0) {
                ++mine;
            } else if (!a.ndrop[w2] && w - w2 > a.excl) {
                Map m{map, map_cap};
                map_add(m, pair_key((uint32_t)(a.first_id + w2), (uint32_t)j), err);
            }
        }
    }
    if (MODE == 0) {
        for (int o = 16; o; o >>= 1) mine += __shfl_down_sync(~0u, mine, o);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
    }
}

// The batch's live windows enter the delta: entry index e0 + w in every table.
__global__ void k_delta_insert(const uint32_t *__restrict__ keys, const uint8_t *__restrict__ ndrop, uint32_t n,
                               uint64_t first_id, uint64_t e0, unsigned long long *__restrict__ dslot, uint64_t cap_k,
                               uint32_t *__restrict__ dent_id, uint32_t *__restrict__ dent_next, uint64_t cap_e,
                               uint32_t *err) {
    const uint32_t t = blockIdx.y;
    unsigned long long *slot = dslot + (uint64_t)t * cap_k;
    uint32_t *did = dent_id + (uint64_t)t * cap_e;
    uint32_t *dnx = dent_next + (uint64_t)t * cap_e;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < n; w += gridDim.x * blockDim.x) {
        if (ndrop[w]) continue;
        const uint32_t key = keys[(uint64_t)t * n + w];
        const uint64_t e = e0 + w;
        did[e] = (uint32_t)(first_id + w);
        const unsigned long long mine_tag = ((unsigned long long)key << 32);
        uint64_t h = dslot_hash(key, cap_k);
        bool done = false;
        for (uint64_t probe = 0; probe < cap_k && !done; probe++) {
            unsigned long long cur = slot[h];
            for (uint32_t spin = 0; spin < 1u << 20; spin++) {  // CAS retries while other windows of the key push
                if (cur == 0) {
                    dnx[e] = 0;
                    __threadfence();
                    const unsigned long long old = atomicCAS(slot + h, 0ull, mine_tag | (e + 1));
                    if (old == 0) {
                        done = true;
                        break;
                    }
                    cur = old;
                }
                if ((cur >> 32) != key) break;  // another key: next slot
                dnx[e] = (uint32_t)cur;         // previous head (+1)
                __threadfence();
                const unsigned long long old = atomicCAS(slot + h, cur, mine_tag | (e + 1));
                if (old == cur) {
                    done = true;
                    break;
                }
                cur = old;
            }
            if (!done && ++h == cap_k) h = 0;
        }
        if (!done) set_err(err, ERR_MAP_FULL);
    }
}

__global__ void k_req_compact(const unsigned long long *__restrict__ slot, uint64_t cap, uint32_t v, uint32_t nbits,
                              unsigned long long *__restrict__ out, unsigned long long *__restrict__ cursor,
                              uint64_t out_cap) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long val = slot[s];
        if (val == 0 || (uint32_t)(val & 0xFF) < v) continue;
        const uint64_t key = val >> 8;
        const uint64_t i = key >> 28, j = key & ((1u << 28) - 1);
        const unsigned long long o = atomicAdd(cursor, 1ull);
        if (out && o < out_cap) out[o] = (i << (nbits + 8)) | (j << 8) | (val & 0xFF);
    }
}

__global__ void k_req_unpack(const unsigned long long *__restrict__ in, uint64_t M, uint32_t nbits,
                             uint32_t *__restrict__ oi, uint32_t *__restrict__ oj, uint8_t *__restrict__ ov) {
    const uint64_t jm = (1ull << nbits) - 1;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = in[x];
        oi[x] = (uint32_t)(k >> (nbits + 8));
        oj[x] = (uint32_t)((k >> 8) & jm);
        ov[x] = (uint8_t)(k & 0xFF);
    }
}

}  // namespace
}  // namespace fastgb

using namespace fastgb;

struct fast_request {
    uint64_t id = 0;
    uint32_t station = 0, n = 0, ld = 0;
    uint64_t first_id = 0;
    std::vector<uint16_t> idx;
    std::mutex mu;
    std::condition_variable cv;
    int state = 0;  // 0 queued, 1 done, 2 failed
    fast_status status = FAST_OK;
    std::string msg;
    std::vector<uint32_t> ri, rj;
    std::vector<uint8_t> rv;
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct fast_station {
    fast_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    fast_tables *hist = nullptr;
    HistGroups hg;
    uint64_t N0 = 0;
    bool loaded = false;
    uint64_t next_id = 0;    // id of the next admitted window
    uint64_t delta_used = 0; // entries used per table
    uint64_t cap_e = 0, cap_k = 0;
    unsigned long long *dslot = nullptr;
    uint32_t *dent_id = nullptr, *dent_next = nullptr;
    uint16_t *h_stage = nullptr;  // pinned staging of one request's input
    size_t h_stage_bytes = 0;
    std::deque<fast_request *> queue;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
};

struct fast_server {
    fast_params p{};
    uint32_t nst = 0;
    uint64_t budget = 0, resident = 0;
    std::atomic<uint64_t> in_flight{0};  // bytes reserved by running requests
    std::mutex adm_mu;
    std::condition_variable adm_cv;
    std::vector<fast_station *> st;
    std::mutex req_mu;
    std::unordered_map<uint64_t, fast_request *> reqs;
    uint64_t next_req = 1;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> fail_at{0};  // host-side fault injection: request id that fails
    std::atomic<uint64_t> admit_ms{300000};  // longest admission wait of one request (ms)
    uint64_t held = 0;                       // budget bytes held by the test hook (under adm_mu)
    int device = 0;
    std::string err;
};

namespace {

uint64_t request_bytes(const fast_params &p, uint32_t n, uint32_t ld) {
    // inputs, keys, sorted keys, ranges, flags, plus a vote map for ~64 candidates per (table, window)
    return (uint64_t)n * ld * 2 + (uint64_t)p.b * n * (4 * 5 + 8) + (uint64_t)n * 8 + (uint64_t)p.b * n * 64 * 16;
}

fast_status process(fast_server *S, fast_station *st, fast_request *r) {
    fast_ctx *c = st->ctx;
    cudaStream_t s = st->stream;
    const fast_params &p = S->p;
    const uint32_t n = r->n, nb = p.b;
    fast_status stt = FAST_OK;
    std::vector<std::pair<void *, size_t>> owned;
    auto alloc = [&](auto **ptr, size_t count) -> fast_status {
        using T = std::remove_reference_t<decltype(**ptr)>;
        fast_status q = dalloc_t(c, ptr, count ? count : 1, s);
        if (!q) owned.push_back({(void *)*ptr, (count ? count : 1) * sizeof(T)});
        return q;
    };
    auto release = [&]() {
        for (auto &o : owned) dfree(c, o.first, o.second, s);
        owned.clear();
    };
    auto fail = [&](fast_status q) {
        release();
        return q;
    };
    if (st->delta_used + n > st->cap_e) return set_error(c, FAST_EBUDGET, "station delta capacity exhausted");
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
    // 1. input and signatures
    const size_t in_bytes = (size_t)n * r->ld * 2;
    if (in_bytes > st->h_stage_bytes) {
        if (st->h_stage) cudaFreeHost(st->h_stage);
        st->h_stage = nullptr;
        if (cudaMallocHost(&st->h_stage, in_bytes) != cudaSuccess) {
            cudaGetLastError();
            st->h_stage_bytes = 0;
            return set_error(c, FAST_ENOMEM, "pinned staging");
        }
        st->h_stage_bytes = in_bytes;
    }
    memcpy(st->h_stage, r->idx.data(), in_bytes);
    uint16_t *d_idx = nullptr;
    uint32_t *keys = nullptr, *bkey = nullptr, *bid = nullptr, *bka = nullptr, *bia = nullptr, *bpos = nullptr,
             *hcnt = nullptr;
    uint2 *range = nullptr;
    uint8_t *ndrop = nullptr;
    uint32_t *wg = nullptr;
    if ((stt = alloc(&wg, (size_t)n * kWG))) return fail(stt);
    if ((stt = alloc(&d_idx, (size_t)n * r->ld)) || (stt = alloc(&keys, (size_t)nb * n)) ||
        (stt = alloc(&bkey, (size_t)nb * n)) || (stt = alloc(&bid, (size_t)nb * n)) ||
        (stt = alloc(&bka, (size_t)nb * n)) || (stt = alloc(&bia, (size_t)nb * n)) ||
        (stt = alloc(&bpos, (size_t)nb * n)) || (stt = alloc(&range, (size_t)nb * n)) || (stt = alloc(&hcnt, n)) ||
        (stt = alloc(&ndrop, n)))
        return fail(stt);
    cudaMemcpyAsync(d_idx, st->h_stage, in_bytes, cudaMemcpyHostToDevice, s);
    if ((stt = sig_launch(c, d_idx, n, r->ld, keys, s))) return fail(stt);
    // 2. history lookup and the frozen filter
    ReqArgs a{};
    a.hkey = st->hist->d_skey;
    a.hid = st->hist->d_sid;
    a.hdrop = st->hist->d_drop;
    a.N0 = st->N0;
    a.dslot = st->dslot;
    a.dent_id = st->dent_id;
    a.dent_next = st->dent_next;
    a.dcap_k = st->cap_k;
    a.dcap_e = st->cap_e;
    a.keys = keys;
    a.n = n;
    a.nb = nb;
    a.excl = p.excl;
    a.first_id = r->first_id;
    a.occ_num = p.occ_num;
    a.occ_den = p.occ_den;
    a.label = st->hg.label;
    a.large = st->hg.large;
    a.tstart = st->hg.tstart;
    a.wg = wg;
    cudaMemsetAsync(wg, 0xFF, (size_t)n * kWG * 4, s);
    cudaMemsetAsync(hcnt, 0, (size_t)n * 4, s);
    const dim3 g(std::max(1u, ceil_div(n, 128)), nb);
    k_req_lookup<<<g, 128, 0, s>>>(a, range, hcnt), FAST_LAUNCHED(c);
    k_req_drop<<<std::max(1u, ceil_div(n, 256)), 256, 0, s>>>(hcnt, n, nb, ndrop), FAST_LAUNCHED(c);
    // 3. the batch's keys sorted per table (earlier same-key windows)
    uint32_t *sk = nullptr, *sv = nullptr;
    if ((stt = sort_u32(c, nb, n, keys, nullptr, bka, bia, bkey, bid, 0, 32, &sk, &sv, s, nullptr))) return fail(stt);
    k_req_inverse<<<g, 128, 0, s>>>(sv, n, bpos), FAST_LAUNCHED(c);
    a.bkey = sk;
    a.bid = sv;
    a.bpos = bpos;
    a.range = range;
    a.ndrop = ndrop;
    // 4. candidate count, vote map
    cudaMemsetAsync(scal, 0, 16, s);
    k_req_pairs<0><<<g, 128, 0, s>>>(a, scal, nullptr, 0, c->d_err), FAST_LAUNCHED(c);
    const bool dense = st->hg.nlarge > 0;
    const size_t dsm = (size_t)nb * 4;
    if (dense)
        k_req_dense<0><<<n, 256, dsm, s>>>(a, st->hg.gstart, st->hg.ids, st->hg.bm, st->hg.bm_off, scal, nullptr, 0,
                                           c->d_err), FAST_LAUNCHED(c);
    uint64_t total = 0;
    cudaMemcpyAsync(&total, scal, 8, cudaMemcpyDeviceToHost, s);
    if ((stt = sync_check(c, s, "request count"))) return fail(stt);
    const uint64_t mcap = std::max<uint64_t>(1024, 2 * total + 1);
    unsigned long long *map = nullptr;
    if ((stt = alloc(&map, mcap))) return fail(stt);
    cudaMemsetAsync(map, 0, mcap * 8, s);
    k_req_pairs<1><<<g, 128, 0, s>>>(a, nullptr, map, mcap, c->d_err), FAST_LAUNCHED(c);
    if (dense)
        k_req_dense<1><<<n, 256, dsm, s>>>(a, st->hg.gstart, st->hg.ids, st->hg.bm, st->hg.bm_off, nullptr, map, mcap,
                                           c->d_err), FAST_LAUNCHED(c);
    // 5. keep, order, copy out
    const uint64_t max_id = r->first_id + n;
    uint32_t nbits = 1;
    while (nbits < 28 && (1ull << nbits) < max_id) nbits++;
    cudaMemsetAsync(scal + 1, 0, 16, s);
    const unsigned cg = (unsigned)std::min<uint64_t>(ceil_div(mcap, 256), c->num_sms * 8);
    k_req_compact<<<cg, 256, 0, s>>>(map, mcap, p.v, nbits, nullptr, scal + 1, 0), FAST_LAUNCHED(c);
    uint64_t Ms = 0, Md = 0;
    cudaMemcpyAsync(&Ms, scal + 1, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&Md, scal + 2, 8, cudaMemcpyDeviceToHost, s);
    if ((stt = sync_check(c, s, "request votes"))) return fail(stt);
    const uint64_t M = Ms + Md;
    r->ri.resize(M);
    r->rj.resize(M);
    r->rv.resize(M);
    if (M) {
        unsigned long long *ok = nullptr, *ok2 = nullptr;
        uint32_t *oi = nullptr, *oj = nullptr;
        uint8_t *ov = nullptr;
        if ((stt = alloc(&ok, M)) || (stt = alloc(&ok2, M)) || (stt = alloc(&oi, M)) || (stt = alloc(&oj, M)) ||
            (stt = alloc(&ov, M)))
            return fail(stt);
        cudaMemsetAsync(scal + 1, 0, 8, s);
        k_req_compact<<<cg, 256, 0, s>>>(map, mcap, p.v, nbits, ok, scal + 1, M), FAST_LAUNCHED(c);

        uint64_t *sorted = reinterpret_cast<uint64_t *>(ok);
        if (M > 1 && (stt = sort_u64(c, M, reinterpret_cast<uint64_t *>(ok), reinterpret_cast<uint64_t *>(ok2), 8,
                                     8 + 2 * nbits, &sorted, s)))
            return fail(stt);
        k_req_unpack<<<std::max(1u, std::min<unsigned>(ceil_div(M, 256), c->num_sms * 8)), 256, 0, s>>>(
            reinterpret_cast<unsigned long long *>(sorted), M, nbits, oi, oj, ov), FAST_LAUNCHED(c);
        cudaMemcpyAsync(r->ri.data(), oi, M * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(r->rj.data(), oj, M * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(r->rv.data(), ov, M, cudaMemcpyDeviceToHost, s);
    }
    // 6. the batch joins the delta (after its own query, in admission order)
    k_delta_insert<<<g, 128, 0, s>>>(keys, ndrop, n, r->first_id, st->delta_used, st->dslot, st->cap_k, st->dent_id,
                                     st->dent_next, st->cap_e, c->d_err), FAST_LAUNCHED(c);
    st->delta_used += n;
    release();
    return sync_check(c, s, "request");
}

// Continuous batching: a worker takes the request at the head of its
// station's queue together with the requests queued right behind it (their
// window ids follow on, admission order), up to kMergeWindows windows, and
// searches them as one batch.  Pair (i, j) then belongs to the request whose
// windows hold j; that request would have found it alone too, because every
// window of the earlier requests precedes j and would have been in the delta.
constexpr uint64_t kMergeWindows = 65536;

void finish(fast_request *r, fast_status res, const std::string &msg) {
    {
        std::lock_guard<std::mutex> lk(r->mu);
        r->status = res;
        r->msg = msg;
        r->state = res ? 2 : 1;
        r->t_done = std::chrono::steady_clock::now();
    }
    r->cv.notify_all();
}

void worker_main(fast_server *S, fast_station *st) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<fast_request *> grp;
        {
            std::unique_lock<std::mutex> lk(st->mu);
            st->cv.wait(lk, [&] { return S->stop.load() || !st->queue.empty(); });
            if (st->queue.empty()) return;  // stopping
            grp.push_back(st->queue.front());
            st->queue.pop_front();
            uint64_t ntot = grp[0]->n;
            while (S->fail_at.load() != grp[0]->id && !st->queue.empty()) {
                fast_request *q = st->queue.front();
                const fast_request *last = grp.back();
                if (q->ld != grp[0]->ld || S->fail_at.load() == q->id || ntot + q->n > kMergeWindows ||
                    q->first_id != last->first_id + last->n)
                    break;
                if (S->budget && S->resident + request_bytes(S->p, (uint32_t)(ntot + q->n), q->ld) > S->budget) break;
                grp.push_back(q);
                st->queue.pop_front();
                ntot += q->n;
            }
        }
        fast_request *r = grp[0];
        fast_request merged;
        fast_request *work = r;
        if (grp.size() > 1) {  // one input, ids from the first request on
            merged.id = r->id;
            merged.station = r->station;
            merged.ld = r->ld;
            merged.first_id = r->first_id;
            for (const fast_request *q : grp) {
                merged.n += q->n;
                merged.idx.insert(merged.idx.end(), q->idx.begin(), q->idx.end());
            }
            work = &merged;
        }
        fast_status res = FAST_OK;
        std::string msg;
        const uint64_t need = request_bytes(S->p, work->n, work->ld);
        if (S->fail_at.load() == r->id) {
            res = FAST_EINTERNAL;  // injected failure
            msg = "injected request failure";
        } else if (S->budget && S->resident + need > S->budget) {
            res = FAST_EBUDGET;
            msg = "request can never fit the HBM budget";
        } else {
            bool admitted = false;
            {   // admission: wait, at most admit_ms, until the request's working
                // set fits next to the running ones
                std::unique_lock<std::mutex> lk(S->adm_mu);
                const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(S->admit_ms.load());
                admitted = S->adm_cv.wait_until(lk, until, [&] {
                    return S->stop.load() || !S->budget || S->resident + S->in_flight.load() + need <= S->budget;
                });
                if (admitted) S->in_flight += need;
            }
            if (!admitted) {
                res = FAST_ETIMEOUT;
                msg = "admission wait ran out: the HBM budget did not free up in time";
            } else {
                if (S->stop.load()) {
                    res = FAST_ETIMEOUT;
                    msg = "server stopped";
                } else {
                    res = process(S, st, work);
                    if (res) msg = st->ctx->err;
                }
                S->in_flight -= need;
                S->adm_cv.notify_all();
            }
        }
        if (grp.size() > 1 && !res) {  // each request takes the pairs whose j lies in its windows
            for (fast_request *q : grp) {
                q->ri.clear();
                q->rj.clear();
                q->rv.clear();
            }
            std::vector<uint64_t> starts;
            for (const fast_request *q : grp) starts.push_back(q->first_id);
            for (size_t e = 0; e < merged.ri.size(); e++) {
                const uint64_t j = merged.rj[e];
                const size_t k = std::upper_bound(starts.begin(), starts.end(), j) - starts.begin() - 1;
                grp[k]->ri.push_back(merged.ri[e]);
                grp[k]->rj.push_back(merged.rj[e]);
                grp[k]->rv.push_back(merged.rv[e]);
            }
        }
        for (fast_request *q : grp) finish(q, res, msg);
    }
}

}  // namespace

extern "C" {

fast_status fast_server_create(const fast_params *p, uint32_t n_stations, uint64_t max_stream_windows,
                               uint64_t hbm_budget_bytes, fast_server **out) {
    if (!out || n_stations == 0 || n_stations > 1024) return FAST_EINVAL;
    *out = nullptr;
    fast_server *S = new fast_server();
    S->p = *p;
    S->nst = n_stations;
    S->budget = hbm_budget_bytes;
    cudaGetDevice(&S->device);
    const uint64_t cap_e = std::max<uint64_t>(max_stream_windows, 1);
    uint64_t cap_k = 2;
    while (cap_k < 2 * cap_e) cap_k <<= 1;
    const uint64_t delta_bytes = (uint64_t)p->b * (cap_k * 8 + cap_e * 8);
    fast_status st = FAST_OK;
    for (uint32_t k = 0; k < n_stations && !st; k++) {
        fast_station *sn = new fast_station();
        S->st.push_back(sn);
        if ((st = fast_create(p, 0, &sn->ctx))) break;
        if (cudaStreamCreateWithFlags(&sn->stream, cudaStreamNonBlocking) != cudaSuccess) {
            st = FAST_ECUDA;
            break;
        }
        sn->cap_e = cap_e;
        sn->cap_k = cap_k;
        if (S->budget && S->resident + delta_bytes > S->budget) {
            st = FAST_EBUDGET;
            S->err = "delta tables do not fit the HBM budget";
            break;
        }
        if (cudaMalloc(&sn->dslot, (size_t)p->b * cap_k * 8) != cudaSuccess ||
            cudaMalloc(&sn->dent_id, (size_t)p->b * cap_e * 4) != cudaSuccess ||
            cudaMalloc(&sn->dent_next, (size_t)p->b * cap_e * 4) != cudaSuccess) {
            cudaGetLastError();
            st = FAST_ENOMEM;
            break;
        }
        cudaMemset(sn->dslot, 0, (size_t)p->b * cap_k * 8);
        S->resident += delta_bytes;
    }
    if (st) {
        fast_server_destroy(S);
        return st;
    }
    for (auto *sn : S->st) sn->worker = std::thread(worker_main, S, sn);
    *out = S;
    return FAST_OK;
}

void fast_server_destroy(fast_server *S) {
    if (!S) return;
    S->stop = true;
    S->adm_cv.notify_all();
    for (auto *sn : S->st) {
        {
            std::lock_guard<std::mutex> lk(sn->mu);
        }
        sn->cv.notify_all();
        if (sn->worker.joinable()) sn->worker.join();
    }
    for (auto *sn : S->st) {
        for (auto *r : sn->queue) {
            std::lock_guard<std::mutex> lk(r->mu);
            r->state = 2;
            r->status = FAST_ETIMEOUT;
        }
        if (sn->stream) cudaStreamSynchronize(sn->stream);
        if (sn->hist) fast_tables_free(sn->hist);
        history_groups_free(&sn->hg);
        if (sn->ctx) fast_destroy(sn->ctx);
        cudaFree(sn->dslot);
        cudaFree(sn->dent_id);
        cudaFree(sn->dent_next);
        if (sn->h_stage) cudaFreeHost(sn->h_stage);
        if (sn->stream) cudaStreamDestroy(sn->stream);
        delete sn;
    }
    for (auto &kv : S->reqs) delete kv.second;
    cudaGetLastError();
    delete S;
}

const char *fast_server_last_error(const fast_server *S) { return S ? S->err.c_str() : "no server"; }

fast_status fast_server_load_history(fast_server *S, uint32_t station, const uint16_t *h_idx, uint64_t N,
                                     uint32_t ld) {
    if (!S || station >= S->nst || (N && !h_idx) || ld < S->p.K) return FAST_EINVAL;
    fast_station *sn = S->st[station];
    std::lock_guard<std::mutex> lk(sn->mu);
    if (sn->loaded || sn->next_id) {
        S->err = "history already loaded or stream started";
        return FAST_EINVAL;
    }
    fast_ctx *c = sn->ctx;
    cudaStream_t s = sn->stream;
    const fast_params &p = S->p;
    const uint64_t hist_bytes = (uint64_t)p.b * N * 8 + N * 5;  // tables, drop mask, labels
    if (S->budget && S->resident + hist_bytes > S->budget) {
        S->err = "history does not fit the HBM budget";
        return FAST_EBUDGET;
    }
    uint16_t *d_idx = nullptr;
    uint32_t *sig = nullptr;
    fast_status st;
    if ((st = dalloc(c, (void **)&d_idx, (size_t)N * ld * 2, s)) ||
        (st = dalloc_t(c, &sig, (size_t)p.b * (N ? N : 1), s))) {
        dfree(c, d_idx, (size_t)N * ld * 2, s);
        S->err = c->err;
        return st;
    }
    cudaMemcpyAsync(d_idx, h_idx, (size_t)N * ld * 2, cudaMemcpyHostToDevice, s);
    st = sig_launch(c, d_idx, N, ld, sig, s);
    fast_tables *tb = nullptr;
    if (!st) st = fast_build_tables(c, sig, N, &tb, s);
    if (!st) st = history_groups(c, tb, sig, &sn->hg, s);
    dfree(c, d_idx, (size_t)N * ld * 2, s);
    dfree(c, sig, (size_t)p.b * (N ? N : 1) * 4, s);
    cudaStreamSynchronize(s);
    if (st) {
        S->err = c->err;
        if (tb) fast_tables_free(tb);
        history_groups_free(&sn->hg);
        return st;
    }
    tb->d_sig = nullptr;  // the server never searches the history itself
    sn->hist = tb;
    sn->N0 = N;
    sn->next_id = N;
    sn->loaded = true;
    S->resident += hist_bytes;
    return FAST_OK;
}

fast_status fast_stream_submit(fast_server *S, uint32_t station, const uint16_t *h_idx, uint32_t n, uint32_t ld,
                               uint64_t *req_id) {
    if (!S || !req_id || station >= S->nst || (n && !h_idx) || ld < S->p.K || n == 0) return FAST_EINVAL;
    fast_station *sn = S->st[station];
    fast_request *r = new fast_request();
    r->station = station;
    r->n = n;
    r->ld = ld;
    r->idx.assign(h_idx, h_idx + (size_t)n * ld);
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S->req_mu);
        r->id = S->next_req++;
        S->reqs[r->id] = r;
    }
    {
        std::lock_guard<std::mutex> lk(sn->mu);
        if (!sn->loaded) {
            std::lock_guard<std::mutex> lk2(S->req_mu);
            S->reqs.erase(r->id);
            delete r;
            S->err = "station has no history";
            return FAST_EINVAL;
        }
        r->first_id = sn->next_id;  // admission order of the station
        sn->next_id += n;
        sn->queue.push_back(r);
    }
    sn->cv.notify_one();
    *req_id = r->id;
    return FAST_OK;
}

fast_status fast_stream_poll(fast_server *S, uint64_t req_id, uint64_t timeout_us, uint64_t *M, uint64_t *first_id,
                             const uint32_t **h_i, const uint32_t **h_j, const uint8_t **h_votes) {
    if (!S) return FAST_EINVAL;
    fast_request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->req_mu);
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return FAST_EINVAL;
        r = it->second;
    }
    std::unique_lock<std::mutex> lk(r->mu);
    if (r->state == 0)
        r->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->state != 0; });
    if (r->state == 0) return FAST_EPENDING;
    if (r->state == 2) {
        S->err = r->msg;
        return r->status;
    }
    if (M) *M = r->ri.size();
    if (first_id) *first_id = r->first_id;
    if (h_i) *h_i = r->ri.data();
    if (h_j) *h_j = r->rj.data();
    if (h_votes) *h_votes = r->rv.data();
    return FAST_OK;
}

fast_status fast_stream_latency(fast_server *S, uint64_t req_id, double *seconds) {
    if (!S || !seconds) return FAST_EINVAL;
    std::lock_guard<std::mutex> lk(S->req_mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return FAST_EINVAL;
    fast_request *r = it->second;
    std::lock_guard<std::mutex> lk2(r->mu);
    if (r->state == 0) return FAST_EPENDING;
    *seconds = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    return FAST_OK;
}

fast_status fast_stream_release(fast_server *S, uint64_t req_id) {
    if (!S) return FAST_EINVAL;
    fast_request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->req_mu);
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return FAST_EINVAL;
        r = it->second;
        {
            std::lock_guard<std::mutex> lk2(r->mu);
            if (r->state == 0) return FAST_EPENDING;
        }
        S->reqs.erase(it);
    }
    delete r;
    return FAST_OK;
}

fast_status fast_server_set_option(fast_server *S, const char *name, double value) {
    if (!S || !name) return FAST_EINVAL;
    if (!strcmp(name, "admit_timeout_ms")) {  // a server setting, allowed at any time
        if (!(value >= 0 && value <= 86400e3)) {
            S->err = "admit_timeout_ms must be in [0, 86400000]";
            return FAST_EINVAL;
        }
        S->admit_ms = (uint64_t)value;
        return FAST_OK;
    }
    for (auto *sn : S->st) {
        std::lock_guard<std::mutex> lk(sn->mu);
        if (sn->loaded) {
            S->err = "options must be set before any history is loaded";
            return FAST_EINVAL;
        }
    }
    for (auto *sn : S->st) {
        fast_status st = fast_set_option(sn->ctx, name, value);
        if (st) {
            S->err = sn->ctx->err;
            return st;
        }
    }
    return FAST_OK;
}

fast_status fast_server_hold_budget(fast_server *S, uint64_t bytes) {
    if (!S) return FAST_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->adm_mu);
        S->in_flight -= S->held;
        S->in_flight += bytes;
        S->held = bytes;
    }
    S->adm_cv.notify_all();
    return FAST_OK;
}

fast_status fast_server_inject_failure(fast_server *S, uint64_t req_id) {
    if (!S) return FAST_EINVAL;
    S->fail_at = req_id;
    return FAST_OK;
}

}  // extern "C"
