// k_query.cu -- query-only hashing (§6.4 "Partition", last paragraph): for a
// small set of new windows queried against a large history, only the new
// windows are put into hash tables; every history window's keys are then
// streamed past those tables, and a key found there gives a vote to each
// (history window, query window) pair in that bucket.  No table of the
// history is built, sorted or filtered -- the paper's cheaper way of running
// a thousand queries on a million items, with results identical to querying
// tables of the whole data set.
//
// Semantics: the batch's windows follow the history on the station
// timeline (ids N0 .. N0 + n - 1), exactly as one streamed request after the
// history: every pair (i, j) with j in the batch and i < j (i in the history
// or in the batch), neither dropped, j - i > excl, votes >= v, sorted by
// (i, j).  History windows carry the caller's drop flags; a batch window is
// dropped when its key falls in a heavy history bucket (occ_den * size >
// occ_num * N0, sizes counted over all N0 history windows) in more than b/2
// tables -- the counts come from the same streaming pass.
//
// GB300 design.  Query tables: the batch's keys sorted per table (radix
// sort, b * n entries).  Probe kernel: a CTA takes a tile of one table's
// history keys (coalesced) and binary-searches each in that table's sorted
// query keys, staged in shared memory when they fit; a first pass counts the
// history members of every query bucket (the heavy test) and the pair votes
// to come (the map's size), a second adds the votes to a device
// open-addressing map of packed (i, j) -> votes.  Pairs inside the batch come
// from runs of equal keys in the query tables.  Kept pairs are compacted and
// ordered by one radix sort of their packed (i, j).
#include <algorithm>
#include <type_traits>

#include "fast_internal.cuh"

namespace fastgb {
namespace {

constexpr uint32_t kQThreads = 256;
constexpr uint32_t kQSmemKeys = 12288;  // query keys of one table staged in shared memory (48 KB)

__device__ __forceinline__ uint32_t lower_key(const uint32_t *k, uint32_t n, uint32_t key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (k[m] < key) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// MODE 0: hsize[t][run start] += 1 per history window with that key, and the
// pair votes to come are counted; MODE 1: the votes are added to the map.
template <int MODE>
__global__ void __launch_bounds__(kQThreads) k_q_probe(const uint32_t *__restrict__ hkey, uint64_t N0,
                                                       const uint8_t *__restrict__ hdrop,
                                                       const uint32_t *__restrict__ qkey,
                                                       const uint32_t *__restrict__ qid, uint32_t n,
                                                       const uint8_t *__restrict__ qdrop, uint32_t excl,
                                                       uint32_t *__restrict__ hsize, unsigned long long *npairs,
                                                       Map map, uint32_t *err) {
    __shared__ uint32_t sk[kQSmemKeys];
    const uint32_t t = blockIdx.y;
    const uint32_t *K = qkey + (uint64_t)t * n;
    const uint32_t *Q = qid + (uint64_t)t * n;
    const bool staged = n <= kQSmemKeys;
    if (staged) {
        for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) sk[x] = K[x];
        __syncthreads();
    }
    const uint32_t *KS = staged ? sk : K;
    unsigned long long mine = 0;
    for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < N0; h += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t key = __ldcs(hkey + (uint64_t)t * N0 + h);
        const uint32_t lo = lower_key(KS, n, key);
        if (lo == n || KS[lo] != key) continue;
        if (MODE == 0) atomicAdd(hsize + (uint64_t)t * n + lo, 1u);
        if (hdrop && hdrop[h]) continue;
        for (uint32_t p = lo; p < n && KS[p] == key; p++) {
            const uint32_t q = Q[p];
            const uint64_t j = N0 + q;
            if (j - h <= excl) continue;
            if (MODE == 0) {
                mine++;
            } else if (!qdrop[q]) {
                map_add(map, pair_key((uint32_t)h, (uint32_t)j), err);
            }
        }
    }
    if (MODE == 0 && mine) atomicAdd(npairs, mine);
}

// Heavy test of the batch windows: for each sorted position p of table t,
// the history bucket size of its key sits at the run's first position.
__global__ void k_q_heavy(const uint32_t *__restrict__ qkey, const uint32_t *__restrict__ qid, uint32_t n,
                          uint32_t nb, const uint32_t *__restrict__ hsize, uint64_t N0, uint32_t occ_num,
                          uint32_t occ_den, uint32_t *__restrict__ heavy) {
    const uint64_t total = (uint64_t)nb * n;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = e / n, p = e % n;
        const uint32_t *K = qkey + t * n;
        const uint32_t r = lower_key(K, n, K[p]);  // first position of p's run
        const uint64_t size = hsize[t * n + r];
        if ((uint64_t)occ_den * size > (uint64_t)occ_num * N0) atomicAdd(heavy + qid[t * n + p], 1u);
    }
}

__global__ void k_q_drop(const uint32_t *__restrict__ heavy, uint32_t n, uint32_t nb, uint32_t occ_num,
                         uint8_t *__restrict__ qdrop) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        qdrop[q] = occ_num > 0 && 2 * heavy[q] > nb;
}

// Pairs inside the batch: positions p < p2 of one run of equal keys.
template <int MODE>
__global__ void k_q_inner(const uint32_t *__restrict__ qkey, const uint32_t *__restrict__ qid, uint32_t n,
                          uint32_t nb, uint64_t N0, const uint8_t *__restrict__ qdrop, uint32_t excl,
                          unsigned long long *npairs, Map map, uint32_t *err) {
    const uint64_t total = (uint64_t)nb * n;
    unsigned long long mine = 0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = e / n, p = e % n;
        const uint32_t *K = qkey + t * n;
        const uint32_t *Q = qid + t * n;
        const uint32_t a = Q[p];
        for (uint64_t p2 = p + 1; p2 < n && K[p2] == K[p]; p2++) {
            const uint32_t b = Q[p2];
            const uint32_t lo = min(a, b), hi = max(a, b);
            if (hi - lo <= excl) continue;
            if (MODE == 0) mine++;
            else if (!qdrop[lo] && !qdrop[hi])
                map_add(map, pair_key((uint32_t)(N0 + lo), (uint32_t)(N0 + hi)), err);
        }
    }
    if (MODE == 0 && mine) atomicAdd(npairs, mine);
}

// Slots with votes >= v, as packed (i:28 | j:28) keys with the votes in the
// low byte, compacted by a warp-aggregated cursor.
__global__ void k_q_compact(const unsigned long long *__restrict__ slot, uint64_t cap, uint32_t v,
                            unsigned long long *__restrict__ out, unsigned long long *cursor) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < cap; x += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned am = __activemask();
        const unsigned long long s = slot[x];
        const bool keep = s != 0 && (s & 0xFF) >= v;
        const unsigned m = __ballot_sync(am, keep);
        if (!m) continue;  // uniform over the threads in am
        const unsigned lane = threadIdx.x & 31, leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(m));
        base = __shfl_sync(am, base, leader);
        if (keep) out[base + __popc(m & ((1u << lane) - 1))] = s;
    }
}

__global__ void k_q_unpack(const unsigned long long *__restrict__ w, uint64_t M, uint32_t *__restrict__ oi,
                           uint32_t *__restrict__ oj, uint8_t *__restrict__ ov) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long s = w[x];
        oi[x] = (uint32_t)(s >> 36);
        oj[x] = (uint32_t)((s >> 8) & ((1u << 28) - 1));
        ov[x] = (uint8_t)(s & 0xFF);
    }
}

unsigned grid_of(const fast_ctx *c, uint64_t n) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)c->num_sms * 8));
}

}  // namespace
}  // namespace fastgb

using namespace fastgb;

extern "C" fast_status fast_query_only(fast_ctx *c, const uint16_t *d_hist, uint64_t N0, const uint8_t *d_hist_drop,
                                       const uint16_t *d_batch, uint64_t n, uint32_t ld, fast_result **out,
                                       void *stream) {
    if (!c || !out) return FAST_EINVAL;
    c->err.clear();
    *out = nullptr;
    const fast_params &p = c->p;
    if ((N0 && !d_hist) || (n && !d_batch) || ld < p.K)
        return set_error(c, FAST_EINVAL, "fast_query_only: bad arguments");
    if (N0 + n >= (1ull << 28)) return set_error(c, FAST_EINVAL, "fast_query_only: N0 + n must be < 2^28");
    cudaStream_t s = (cudaStream_t)stream;
    c->stats.n_launches = 0;
    const uint32_t nb = p.b, nq = (uint32_t)n;
    std::vector<std::pair<void *, size_t>> owned;
    auto alloc = [&](auto **ptr, size_t count) -> fast_status {
        using T = std::remove_reference_t<decltype(**ptr)>;
        fast_status r = dalloc_t(c, ptr, count ? count : 1, s);
        if (!r) owned.push_back({(void *)*ptr, (count ? count : 1) * sizeof(T)});
        return r;
    };
    auto release = [&]() {
        for (auto &o : owned) dfree(c, o.first, o.second, s);
        owned.clear();
    };
    fast_result *res = new fast_result();
    res->ctx = c;
    res->stream = s;
    auto fail_res = [&](fast_status r) {
        release();
        fast_result_free(res);
        return r;
    };
    fast_status st;
    // ---- keys: the batch (then its tables) and the history (streamed)
    uint32_t *hkey = nullptr, *bkey = nullptr, *ka = nullptr, *va = nullptr, *qk = nullptr, *qi = nullptr;
    const size_t nbn = (size_t)nb * n, nbh = (size_t)nb * N0;
    if ((st = alloc(&hkey, nbh)) || (st = alloc(&bkey, nbn)) || (st = alloc(&ka, nbn)) || (st = alloc(&va, nbn)) ||
        (st = alloc(&qk, nbn)) || (st = alloc(&qi, nbn)))
        return fail_res(st);
    if ((st = sig_launch(c, d_hist, N0, ld, hkey, s)) || (st = sig_launch(c, d_batch, n, ld, bkey, s)))
        return fail_res(st);
    uint32_t *ko = nullptr, *vo = nullptr;
    if ((st = sort_u32(c, nb, n, bkey, nullptr, ka, va, qk, qi, 0, 32, &ko, &vo, s, nullptr))) return fail_res(st);
    // ---- pass 1: history bucket sizes of the batch keys, pair counts, the heavy test
    uint32_t *hsize = nullptr, *heavy = nullptr;
    uint8_t *qdrop = nullptr;
    if ((st = alloc(&hsize, nbn)) || (st = alloc(&heavy, n)) || (st = alloc(&qdrop, n))) return fail_res(st);
    cudaMemsetAsync(hsize, 0, nbn * 4, s);
    cudaMemsetAsync(heavy, 0, (size_t)n * 4, s);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c->d_scal);
    cudaMemsetAsync(cnt, 0, 16, s);
    const dim3 pg((unsigned)std::max<uint64_t>(1, std::min<uint64_t>((N0 + kQThreads - 1) / kQThreads,
                                                                     std::max<uint64_t>(1, c->num_sms * 16 / nb))),
                  nb);
    Map none{nullptr, 0};
    if (N0 && n)
        k_q_probe<0><<<pg, kQThreads, 0, s>>>(hkey, N0, d_hist_drop, ko, vo, nq, nullptr, p.excl, hsize, cnt, none,
                                              c->d_err), FAST_LAUNCHED(c);
    if (n) {
        k_q_heavy<<<grid_of(c, nbn), 256, 0, s>>>(ko, vo, nq, nb, hsize, N0, p.occ_num, p.occ_den, heavy),
            FAST_LAUNCHED(c);
        k_q_drop<<<grid_of(c, n), 256, 0, s>>>(heavy, nq, nb, p.occ_num, qdrop), FAST_LAUNCHED(c);
        k_q_inner<0><<<grid_of(c, nbn), 256, 0, s>>>(ko, vo, nq, nb, N0, qdrop, p.excl, cnt + 1, none, c->d_err),
            FAST_LAUNCHED(c);
    }
    cudaMemcpyAsync(c->h_scal, cnt, 16, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "query-only count"))) return fail_res(st);
    const uint64_t pairs = c->h_scal[0] + c->h_scal[1];
    // ---- pass 2: votes into an open-addressing map of packed (i, j) -> votes
    uint64_t cap = 1024;
    while ((double)cap * c->map_load < (double)pairs) cap <<= 1;
    unsigned long long *slot = nullptr;
    if ((st = alloc(&slot, cap))) return fail_res(st);
    cudaMemsetAsync(slot, 0, cap * 8, s);
    const Map map{slot, cap};
    if (N0 && n)
        k_q_probe<1><<<pg, kQThreads, 0, s>>>(hkey, N0, d_hist_drop, ko, vo, nq, qdrop, p.excl, nullptr, nullptr, map,
                                              c->d_err), FAST_LAUNCHED(c);
    if (n)
        k_q_inner<1><<<grid_of(c, nbn), 256, 0, s>>>(ko, vo, nq, nb, N0, qdrop, p.excl, nullptr, map, c->d_err),
            FAST_LAUNCHED(c);
    // ---- kept pairs in (i, j) order
    unsigned long long *kept = nullptr, *kept2 = nullptr;
    const uint64_t kcap = std::min<uint64_t>(cap, pairs + 1);
    if ((st = alloc(&kept, kcap)) || (st = alloc(&kept2, kcap))) return fail_res(st);
    cudaMemsetAsync(cnt + 2, 0, 8, s);
    k_q_compact<<<grid_of(c, cap), 256, 0, s>>>(slot, cap, p.v, kept, cnt + 2), FAST_LAUNCHED(c);
    cudaMemcpyAsync(c->h_scal + 2, cnt + 2, 8, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "query-only votes"))) return fail_res(st);
    const uint64_t M = c->h_scal[2];
    uint64_t *sorted = nullptr;
    if ((st = sort_u64(c, M, reinterpret_cast<uint64_t *>(kept), reinterpret_cast<uint64_t *>(kept2), 8, 64, &sorted,
                       s)))
        return fail_res(st);
    res->M = M;
    const uint64_t m1 = M ? M : 1;
    if ((st = dalloc_t(c, &res->d_i, m1, s)) || (st = dalloc_t(c, &res->d_j, m1, s)) ||
        (st = dalloc_t(c, &res->d_votes, m1, s)))
        return fail_res(st);
    if (M)
        k_q_unpack<<<grid_of(c, M), 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(sorted), M, res->d_i,
                                                 res->d_j, res->d_votes), FAST_LAUNCHED(c);
    release();
    if ((st = sync_check(c, s, "query-only output"))) {
        fast_result_free(res);
        return st;
    }
    c->stats.n_emissions = pairs;
    c->stats.n_detections = M;
    c->stats.map_slots = cap;
    *out = res;
    return FAST_OK;
}
