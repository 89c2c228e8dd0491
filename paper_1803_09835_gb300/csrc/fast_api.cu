// fast_api.cu -- the C-ABI entry points (include/fast.h), the context's
// stream-ordered memory pool with its HBM budget, error plumbing and stage
// timers.  Every step of the search runs in the kernels of k_sig.cu,
// k_sort.cu and k_search.cu; this file only validates, allocates and
// sequences them.
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "fast_internal.cuh"

using namespace fastgb;

namespace fastgb {

fast_status set_error(fast_ctx *c, fast_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

fast_status cuda_fail(fast_ctx *c, cudaError_t e, const char *where) {
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return set_error(c, e == cudaErrorMemoryAllocation ? FAST_ENOMEM : FAST_ECUDA, m);
}

fast_status dalloc(fast_ctx *c, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    const size_t rounded = (bytes + 255) & ~(size_t)255;
    if (c->trace) c->trace_total += rounded;
    if (c->arena) {
        if (c->arena_off + rounded > c->arena_size) return set_error(c, FAST_EINTERNAL, "plan arena exhausted");
        *p = c->arena + c->arena_off;
        c->arena_off += rounded;
        return FAST_OK;
    }
    if (c->budget && c->live + bytes > c->budget)
        return set_error(c, FAST_EBUDGET,
                         "HBM budget exceeded: " + std::to_string(c->live + bytes) + " > " + std::to_string(c->budget));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, s);
    if (e == cudaErrorMemoryAllocation && !c->capturing) {
        // the pool's cached blocks may be free but too fragmented for this
        // request: give them back to the driver and try once more
        cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaMemPoolTrimTo(c->pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes, c->pool, s);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        const std::string what = "device allocation of " + std::to_string(bytes) + " bytes (" +
                                 std::to_string(c->live) + " held, after stage mark " +
                                 std::to_string(c->last_stage) + ")";
        return cuda_fail(c, e, what.c_str());
    }
    c->live += bytes;
    c->peak = std::max(c->peak, c->live);
    return FAST_OK;
}

void dfree(fast_ctx *c, void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (c->arena && (char *)p >= c->arena && (char *)p < c->arena + c->arena_size) return;  // arena: freed with the plan
    if (bytes == 0) bytes = 16;
    cudaFreeAsync(p, s);
    c->live -= std::min<uint64_t>(c->live, bytes);
}

fast_status sync_check(fast_ctx *c, cudaStream_t s, const char *where) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(c, e, where);
    uint32_t flags = 0;
    e = cudaMemcpy(&flags, c->d_err, 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(c, e, where);
    if (!flags) return FAST_OK;
    cudaMemset(c->d_err, 0, 4);
    std::string w(where);
    if (flags & ERR_BAD_INDEX) return set_error(c, FAST_EINVAL, w + ": fingerprint index >= D");
    if (flags & ERR_WALK) return set_error(c, FAST_EINVAL, w + ": fingerprint with no valid index");
    if (flags & ERR_MAP_FULL) return set_error(c, FAST_EMAPFULL, w + ": vote map probe limit reached");
    if (flags & ERR_OVERFLOW) return set_error(c, FAST_EINTERNAL, w + ": device list capacity exceeded");
    if (flags & ERR_INPUT) return set_error(c, FAST_EINVAL, w + ": input list out of order or out of range");
    return set_error(c, FAST_EINTERNAL, w + ": device error flag " + std::to_string(flags));
}

void sig_release(fast_ctx *c, cudaStream_t s) {
    if (!c->sig_owned) return;
    dfree(c, c->sig_owned, c->sig_owned_bytes, s);
    c->sig_owned = nullptr;
    c->sig_owned_bytes = 0;
}

static thread_local uint32_t g_marked = 0;  // stage slots recorded by the current call on this thread

void stage_reset() { g_marked = 0; }

void stage_mark(fast_ctx *c, int slot, cudaStream_t s) {
    c->last_stage = slot;
    if (!c->timing || c->capturing) return;
    cudaEventRecord(c->ev[slot], s);
    g_marked |= 1u << slot;
}

float stage_ms(fast_ctx *c, int a, int b) {
    if (!c->timing || !(g_marked >> a & 1) || !(g_marked >> b & 1)) return 0.f;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

}  // namespace fastgb

static fast_status validate(const fast_params *p, std::string &why) {
    if (!p) return why = "params is NULL", FAST_EINVAL;
    if (p->D < 1 || p->D > 65536) return why = "D must be in [1, 65536]", FAST_EINVAL;
    if (p->K < 1 || p->K > p->D) return why = "K must be in [1, D]", FAST_EINVAL;
    if (p->b < 1 || p->b > 255) return why = "b must be in [1, 255]", FAST_EINVAL;
    if (p->r < 1 || p->r > 16) return why = "r must be in [1, 16]", FAST_EINVAL;
    if (p->kind != FAST_MINHASH && p->kind != FAST_MINMAX) return why = "unknown hash kind", FAST_EINVAL;
    if (p->v < 1 || p->v > p->b) return why = "v must be in [1, b]", FAST_EINVAL;
    if (p->occ_num > 0 && p->occ_den == 0) return why = "occ_den must be > 0 when the filter is on", FAST_EINVAL;
    if (p->query_part > 64) return why = "query_part must be <= 64", FAST_EINVAL;
    if (p->table_group > p->b) return why = "table_group must be <= b (0 = all b tables)", FAST_EINVAL;
    return FAST_OK;
}

void stats_times(fast_ctx *c, bool whole) {
    fast_stats &s = c->stats;
    s.ms_sig = whole ? stage_ms(c, 0, 1) : 0.f;
    s.ms_sort = whole ? stage_ms(c, 1, 2) : 0.f;
    s.ms_filter = whole ? stage_ms(c, 2, 9) : 0.f;
    s.ms_enum = stage_ms(c, 3, 4);
    s.ms_dense = stage_ms(c, 4, 5);
    s.ms_sparse = stage_ms(c, 5, 6);
    s.ms_output = stage_ms(c, 6, 8);
    s.ms_total = whole ? stage_ms(c, 0, 8) : stage_ms(c, 3, 8);
    s.ms_pair_count = stage_ms(c, 5, 10);
    s.ms_pair_emit = stage_ms(c, 10, 11);
    s.ms_vote = stage_ms(c, 11, 6);
}

// Tables and search over keys already in d_sig ([b][N]); the rest of fast_detect.
static fast_status detect_from_sig(fast_ctx *c, const uint32_t *sig, uint64_t N, fast_result **out, cudaStream_t s) {
    fast_tables *tb = nullptr;
    fast_status st = build_tables(c, sig, N, nullptr, 1, &tb, s);  // synchronises: reports bad indices too
    if (!st) st = search_run(c, tb, sig, out, s);
    fast_tables_free(tb);
    return st;
}

extern "C" {

fast_status fast_create(const fast_params *p, uint64_t hbm_budget_bytes, fast_ctx **out) {
    if (!out) return FAST_EINVAL;
    *out = nullptr;
    std::string why;
    if (validate(p, why)) return FAST_EINVAL;
    int dev = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return FAST_ECUDA;
    }
    cudaGetDevice(&dev);
    fast_ctx *c = new fast_ctx();
    c->p = *p;
    c->device = dev;
    c->budget = hbm_budget_bytes;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&c->pool, &props);
    if (e) {
        fast_status st = cuda_fail(c, e, "cudaMemPoolCreate");
        delete c;
        return st;
    }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if ((e = cudaMalloc(&c->d_err, 4)) || (e = cudaMemset(c->d_err, 0, 4)) ||
        (e = cudaMalloc(&c->d_scal, sizeof(uint64_t) * kScal)) ||
        (e = cudaMallocHost(&c->h_scal, sizeof(uint64_t) * kScal))) {
        fast_status st = cuda_fail(c, e, "fast_create");
        fast_destroy(c);
        return st;
    }
    for (auto &ev : c->ev) cudaEventCreate(&ev);
    fast_status st = sig_setup(c);
    if (st) {
        fast_destroy(c);
        return st;
    }
    *out = c;
    return FAST_OK;
}

void fast_destroy(fast_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    cudaFree(c->d_a);
    cudaFree(c->d_b);
    cudaFree(c->d_zinit);
    cudaFree(c->d_walk);
    cudaFree(c->d_err);
    cudaFree(c->d_scal);
    if (c->h_scal) cudaFreeHost(c->h_scal);
    for (auto &ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto &ev : c->cev)
        if (ev) cudaEventDestroy(ev);
    for (auto &ev : c->chev)
        if (ev) cudaEventDestroy(ev);
    for (auto *h : c->h_stage)
        if (h) cudaFreeHost(h);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    cudaGetLastError();
    delete c;
}

const char *fast_last_error(const fast_ctx *c) { return c ? c->err.c_str() : "no context"; }

fast_status fast_sig(fast_ctx *c, const uint16_t *d_idx, uint64_t N, uint32_t ld, uint32_t *d_sig, void *stream) {
    if (!c) return FAST_EINVAL;
    c->err.clear();
    if ((N && (!d_idx || !d_sig)) || ld < c->p.K) return set_error(c, FAST_EINVAL, "fast_sig: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    c->stats.n_launches = 0;
    fast_status st = sig_launch(c, d_idx, N, ld, d_sig, s);
    if (st) return st;
    return sync_check(c, s, "fast_sig");
}

fast_status fast_sig_rows(fast_ctx *c, const uint16_t *d_idx, uint64_t n, uint32_t ld, uint32_t *d_sig, uint64_t N,
                          uint64_t col0, void *stream) {
    if (!c) return FAST_EINVAL;
    c->err.clear();
    if ((n && (!d_idx || !d_sig)) || ld < c->p.K || col0 > N || n > N - col0)
        return set_error(c, FAST_EINVAL, "fast_sig_rows: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    fast_status st = sig_launch_rows(c, d_idx, n, ld, d_sig + col0, N, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(c, e, "fast_sig_rows") : FAST_OK;
}

}  // extern "C"

// Builds the tables of N windows; with nst > 1 stations (offsets h_soff,
// nst + 1 entries) the per-table listing is ordered by (station, key, id).
fast_status build_tables(fast_ctx *c, const uint32_t *d_sig, uint64_t N, const uint64_t *h_soff, uint32_t nst,
                         fast_tables **out, cudaStream_t s) {
    *out = nullptr;
    if (N > (1ull << 28) - 1) return set_error(c, FAST_EINVAL, "N must be < 2^28");
    if (N && !d_sig) return set_error(c, FAST_EINVAL, "d_sig is NULL");
    if (nst < 1 || nst > 256) return set_error(c, FAST_EINVAL, "1 to 256 stations per batch");
    const uint32_t nb = c->p.b;
    fast_tables *tb = new fast_tables();
    tb->ctx = c;
    tb->N = N;
    tb->b = nb;
    tb->d_sig = d_sig;
    tb->stream = s;
    tb->nst = nst;
    if (h_soff) tb->soff.assign(h_soff, h_soff + nst + 1);
    else tb->soff = {0, N};
    const size_t n = (size_t)nb * N;
    // table groups (§6.4 "Partition"): the tables are sorted `grp` at a time
    // into their final place, so the sort's scratch pair holds grp * N
    // entries instead of b * N; every group's sorted tables are kept
    const uint32_t grp = c->p.table_group && c->p.table_group < nb ? c->p.table_group : nb;
    const size_t ns = (size_t)grp * N;
    uint32_t *ka = nullptr, *va = nullptr;
    fast_status st;
    if ((st = dalloc_t(c, &tb->d_soff, nst + 1, s)) || (st = dalloc_t(c, &tb->d_skey, n, s)) ||
        (st = dalloc_t(c, &tb->d_sid, n, s)) || (st = dalloc_t(c, &tb->d_drop, N ? N : 1, s)) ||
        (st = dalloc_t(c, &ka, ns, s)) || (st = dalloc_t(c, &va, ns, s))) {
        dfree(c, ka, ns * 4, s);
        dfree(c, va, ns * 4, s);
        fast_tables_free(tb);
        return st;
    }
    if (!c->capturing)  // a captured build gets its offsets uploaded once by the plan
        cudaMemcpyAsync(tb->d_soff, tb->soff.data(), (nst + 1) * 8, cudaMemcpyHostToDevice, s);
    c->stats.sort_passes = 0;
    // several stations: every station's part of a table is sorted on its own
    uint64_t smax = 0;
    for (uint32_t x = 0; x < nst; x++) smax = std::max<uint64_t>(smax, tb->soff[x + 1] - tb->soff[x]);
    const Stations S = nst > 1 ? Stations{tb->d_soff, nst} : Stations{nullptr, 1};
    for (uint32_t t0 = 0; t0 < nb && !st && N; t0 += grp) {
        const uint32_t gn = std::min(grp, nb - t0);
        const size_t off = (size_t)t0 * N, m = (size_t)gn * N;
        uint32_t *dk = tb->d_skey + off, *dv = tb->d_sid + off;
        uint32_t *ko = nullptr, *vo = nullptr;
        st = sort_u32(c, gn, N, d_sig + off, nullptr, ka, va, dk, dv, 0, 32, &ko, &vo, s, &c->stats.sort_passes, S,
                      smax);
        if (!st && ko != dk) {  // odd number of passes: result sits in the scratch pair
            cudaMemcpyAsync(dk, ko, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(dv, vo, m * 4, cudaMemcpyDeviceToDevice, s);
        }
    }
    dfree(c, ka, ns * 4, s);
    dfree(c, va, ns * 4, s);
    stage_mark(c, 2, s);
    if (!st) st = filter_launch(c, tb, s);
    stage_mark(c, 9, s);
    if (st) {
        fast_tables_free(tb);
        return st;
    }
    *out = tb;
    return FAST_OK;
}

extern "C" {

fast_status fast_build_tables(fast_ctx *c, const uint32_t *d_sig, uint64_t N, fast_tables **out, void *stream) {
    if (!c || !out) return FAST_EINVAL;
    c->err.clear();
    c->stats.n_launches = 0;
    return build_tables(c, d_sig, N, nullptr, 1, out, (cudaStream_t)stream);
}

fast_status fast_tables_view(const fast_tables *tb, uint64_t *N, uint32_t *b, const uint32_t **d_skey,
                             const uint32_t **d_sid, const uint8_t **d_drop) {
    if (!tb) return FAST_EINVAL;
    if (N) *N = tb->N;
    if (b) *b = tb->b;
    if (d_skey) *d_skey = tb->d_skey;
    if (d_sid) *d_sid = tb->d_sid;
    if (d_drop) *d_drop = tb->d_drop;
    return FAST_OK;
}

void fast_tables_free(fast_tables *tb) {
    if (!tb) return;
    fast_ctx *c = tb->ctx;
    const size_t n = (size_t)tb->b * tb->N;
    dfree(c, tb->d_skey, n * 4, tb->stream);
    dfree(c, tb->d_sid, n * 4, tb->stream);
    dfree(c, tb->d_drop, tb->N ? tb->N : 1, tb->stream);
    dfree(c, tb->d_soff, (tb->nst + 1) * 8, tb->stream);
    dfree(c, tb->d_big, tb->big_cap * sizeof(uint4), tb->stream);
    dfree(c, tb->d_bigcnt, 16, tb->stream);
    delete tb;
}

fast_status fast_search(fast_ctx *c, const fast_tables *tb, fast_result **out, void *stream) {
    if (!c || !tb || !out || tb->ctx != c) return FAST_EINVAL;
    c->err.clear();
    *out = nullptr;
    g_marked = 0;
    c->stats.n_launches = 0;
    cudaStream_t s = (cudaStream_t)stream;
    fast_status st = search_run(c, tb, tb->d_sig, out, s);
    if (!st) stats_times(c, false);
    return st;
}

fast_status fast_detect(fast_ctx *c, const uint16_t *d_idx, uint64_t N, uint32_t ld, fast_result **out,
                        void *stream) {
    if (!c || !out) return FAST_EINVAL;
    c->err.clear();
    *out = nullptr;
    if ((N && !d_idx) || ld < c->p.K) return set_error(c, FAST_EINVAL, "fast_detect: bad arguments");
    if (N > (1ull << 28) - 1) return set_error(c, FAST_EINVAL, "N must be < 2^28");
    cudaStream_t s = (cudaStream_t)stream;
    g_marked = 0;
    c->stats.n_launches = 0;
    c->peak = c->live;
    stage_mark(c, 0, s);
    uint32_t *sig = nullptr;
    const size_t n = (size_t)c->p.b * N;
    fast_status st = dalloc_t(c, &sig, n ? n : 1, s);
    if (st) return st;
    c->sig_owned = sig;
    c->sig_owned_bytes = (n ? n : 1) * 4;
    st = sig_launch(c, d_idx, N, ld, sig, s);
    stage_mark(c, 1, s);
    if (!st) st = detect_from_sig(c, sig, N, out, s);
    sig_release(c, s);
    if (!st) stats_times(c, true);
    c->stats.n_fingerprints = N;
    c->stats.peak_bytes = c->peak;
    return st;
}

// Splits a batch's (i, j)-ordered list into per-station lists with local ids.
__global__ void k_split_station(const uint32_t *__restrict__ gi, const uint32_t *__restrict__ gj,
                                const uint8_t *__restrict__ gv, uint64_t a0, uint64_t m, uint32_t base,
                                uint32_t *__restrict__ oi, uint32_t *__restrict__ oj, uint8_t *__restrict__ ov) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < m; x += (uint64_t)gridDim.x * blockDim.x) {
        oi[x] = gi[a0 + x] - base;
        oj[x] = gj[a0 + x] - base;
        ov[x] = gv[a0 + x];
    }
}

__global__ void k_station_bounds(const uint32_t *__restrict__ gi, uint64_t M, const uint64_t *__restrict__ soff,
                                 uint32_t nst, unsigned long long *__restrict__ first) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nst) return;
    uint64_t lo = 0, hi = M;  // first entry with i >= soff[s]
    while (lo < hi) {
        const uint64_t m = (lo + hi) / 2;
        if (gi[m] < soff[s]) lo = m + 1;
        else hi = m;
    }
    first[s] = lo;
}

}  // extern "C"

namespace fastgb {
// Splits a batch result (global ids, (i, j) order) into per-station results
// with local ids; frees `all`.
fast_status split_stations(fast_ctx *c, fast_result *all, const std::vector<uint64_t> &soff, fast_result **out,
                           cudaStream_t s) {
    const uint32_t n_st = (uint32_t)soff.size() - 1;
    if (n_st == 1) {  // one station: its ids are already local
        out[0] = all;
        return FAST_OK;
    }
    unsigned long long *first = nullptr;
    uint64_t *d_soff = nullptr;
    fast_status st;
    if ((st = dalloc_t(c, &first, n_st + 1, s)) || (st = dalloc_t(c, &d_soff, n_st + 1, s))) {
        fast_result_free(all);
        return st;
    }
    cudaMemcpyAsync(d_soff, soff.data(), (n_st + 1) * 8, cudaMemcpyHostToDevice, s);
    k_station_bounds<<<ceil_div(n_st + 1, 128), 128, 0, s>>>(all->d_i, all->M, d_soff, n_st, first), FAST_LAUNCHED(c);
    std::vector<unsigned long long> hf(n_st + 1);
    cudaMemcpyAsync(hf.data(), first, (n_st + 1) * 8, cudaMemcpyDeviceToHost, s);
    st = sync_check(c, s, "station bounds");
    hf[n_st] = all->M;
    for (uint32_t x = 0; x < n_st && !st; x++) {
        fast_result *r = new fast_result();
        r->ctx = c;
        r->stream = s;
        r->M = hf[x + 1] - hf[x];
        const uint64_t m = r->M ? r->M : 1;
        if ((st = dalloc_t(c, &r->d_i, m, s)) || (st = dalloc_t(c, &r->d_j, m, s)) ||
            (st = dalloc_t(c, &r->d_votes, m, s))) {
            fast_result_free(r);
            break;
        }
        if (r->M)
            k_split_station<<<std::max(1u, std::min<unsigned>(ceil_div(r->M, 256), c->num_sms * 8)), 256, 0, s>>>(
                all->d_i, all->d_j, all->d_votes, hf[x], r->M, (uint32_t)soff[x], r->d_i, r->d_j, r->d_votes),
                FAST_LAUNCHED(c);
        out[x] = r;
    }
    dfree(c, first, (n_st + 1) * 8, s);
    dfree(c, d_soff, (n_st + 1) * 8, s);
    fast_result_free(all);
    if (!st) st = sync_check(c, s, "batch split");
    if (st)
        for (uint32_t x = 0; x < n_st; x++) {
            fast_result_free(out[x]);
            out[x] = nullptr;
        }
    return st;
}
}  // namespace fastgb

extern "C" {

fast_status fast_detect_batch(fast_ctx *c, const uint16_t *d_idx, const uint64_t *h_station_N, uint32_t n_st,
                              uint32_t ld, fast_result **out, void *stream) {
    if (!c || !out || !h_station_N || n_st == 0) return FAST_EINVAL;
    c->err.clear();
    for (uint32_t x = 0; x < n_st; x++) out[x] = nullptr;
    if (n_st > 256) return set_error(c, FAST_EINVAL, "at most 256 stations per batch");
    if (ld < c->p.K) return set_error(c, FAST_EINVAL, "ld < K");
    std::vector<uint64_t> soff(n_st + 1, 0);
    for (uint32_t x = 0; x < n_st; x++) soff[x + 1] = soff[x] + h_station_N[x];
    const uint64_t N = soff[n_st];
    if (N > (1ull << 28) - 1) return set_error(c, FAST_EINVAL, "batch larger than 2^28 - 1 windows");
    if (N && !d_idx) return set_error(c, FAST_EINVAL, "d_idx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    g_marked = 0;
    c->stats.n_launches = 0;
    c->peak = c->live;
    stage_mark(c, 0, s);
    uint32_t *sig = nullptr;
    const size_t n = (size_t)c->p.b * N;
    fast_status st = dalloc_t(c, &sig, n ? n : 1, s);
    if (st) return st;
    c->sig_owned = sig;
    c->sig_owned_bytes = (n ? n : 1) * 4;
    st = sig_launch(c, d_idx, N, ld, sig, s);
    stage_mark(c, 1, s);
    fast_tables *tb = nullptr;
    fast_result *all = nullptr;
    if (!st) st = build_tables(c, sig, N, soff.data(), n_st, &tb, s);
    if (!st) st = search_run(c, tb, sig, &all, s);
    fast_tables_free(tb);
    sig_release(c, s);
    if (st) return st;
    if ((st = split_stations(c, all, soff, out, s))) return st;
    stats_times(c, true);
    c->stats.n_fingerprints = N;
    return FAST_OK;
}

fast_status fast_detect_host(fast_ctx *c, const uint16_t *h_idx, uint64_t N, uint32_t ld, uint64_t *M,
                             uint32_t *h_i, uint32_t *h_j, uint8_t *h_votes, uint64_t cap, void *stream) {
    if (!c || !M || (N && !h_idx) || (cap && (!h_i || !h_j || !h_votes))) return FAST_EINVAL;
    c->err.clear();
    if (ld < c->p.K) return set_error(c, FAST_EINVAL, "fast_detect_host: ld < K");
    if (N > (1ull << 28) - 1) return set_error(c, FAST_EINVAL, "N must be < 2^28");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (!c->copy_stream) {
        if ((e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking))) return cuda_fail(c, e, "copy stream");
        for (auto &ev : c->cev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return cuda_fail(c, e, "copy events");
    }
    g_marked = 0;
    c->stats.n_launches = 0;
    stage_mark(c, 0, s);
    uint16_t *d_idx = nullptr;
    uint32_t *sig = nullptr;
    const size_t bytes = (size_t)N * ld * 2, nsig = (size_t)c->p.b * N;
    fast_status st = dalloc(c, (void **)&d_idx, bytes, s);
    if (st) return st;
    if ((st = dalloc_t(c, &sig, nsig ? nsig : 1, s))) {
        dfree(c, d_idx, bytes, s);
        return st;
    }
    c->sig_owned = sig;
    c->sig_owned_bytes = (nsig ? nsig : 1) * 4;
    // chunks of whole 32-row tiles: chunk k is copied on the copy stream while
    // the signature kernel works on chunk k - 1
    const uint64_t per = std::max<uint64_t>(32, ((N + kCopyChunks - 1) / kCopyChunks + 31) / 32 * 32);
    cudaEventRecord(c->cev[kCopyChunks], s);  // the buffers' allocations, ordered on s
    cudaStreamWaitEvent(c->copy_stream, c->cev[kCopyChunks], 0);
    for (uint64_t r0 = 0, k = 0; r0 < N && !st; r0 += per, k++) {
        const uint64_t rows = std::min<uint64_t>(per, N - r0);
        cudaMemcpyAsync(d_idx + r0 * ld, h_idx + r0 * ld, rows * ld * 2, cudaMemcpyHostToDevice, c->copy_stream);
        cudaEventRecord(c->cev[k], c->copy_stream);
        cudaStreamWaitEvent(s, c->cev[k], 0);
        st = sig_launch_rows(c, d_idx + r0 * ld, rows, ld, sig + r0, N, s);
    }
    stage_mark(c, 1, s);
    fast_result *res = nullptr;
    if (!st) st = detect_from_sig(c, sig, N, &res, s);
    sig_release(c, s);
    dfree(c, d_idx, bytes, s);
    if (st) return st;
    stats_times(c, true);
    c->stats.n_fingerprints = N;
    *M = res->M;
    const uint64_t m = std::min<uint64_t>(cap, res->M);
    if (m) {
        cudaMemcpyAsync(h_i, res->d_i, m * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h_j, res->d_j, m * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h_votes, res->d_votes, m, cudaMemcpyDeviceToHost, s);
    }
    st = sync_check(c, s, "fast_detect_host copy-out");
    fast_result_free(res);
    return st;
}

fast_status fast_detect_chunked(fast_ctx *c, uint64_t N, uint32_t ld, uint64_t chunk_rows, fast_fill_rows fill,
                                void *user, fast_result **out, void *stream) {
    if (!c || !out) return FAST_EINVAL;
    c->err.clear();
    *out = nullptr;
    if (!fill || ld < c->p.K || chunk_rows == 0) return set_error(c, FAST_EINVAL, "fast_detect_chunked: bad arguments");
    if (N > (1ull << 28) - 1) return set_error(c, FAST_EINVAL, "N must be < 2^28");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (!c->copy_stream && (e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)))
        return cuda_fail(c, e, "copy stream");
    for (auto &ev : c->chev)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return cuda_fail(c, e, "chunk events");
    chunk_rows = std::min<uint64_t>(chunk_rows, std::max<uint64_t>(N, 1));
    const size_t cbytes = (size_t)chunk_rows * ld * 2;
    if (c->h_stage_bytes < cbytes) {  // pinned staging, kept for later calls
        for (auto *&h : c->h_stage) {
            if (h) cudaFreeHost(h);
            h = nullptr;
        }
        c->h_stage_bytes = 0;
        for (auto *&h : c->h_stage)
            if ((e = cudaMallocHost(&h, cbytes))) return cuda_fail(c, e, "pinned staging");
        c->h_stage_bytes = cbytes;
    }
    g_marked = 0;
    c->stats.n_launches = 0;
    c->peak = c->live;
    stage_mark(c, 0, s);
    uint32_t *sig = nullptr;
    uint16_t *d_chunk[2] = {};
    const size_t nsig = (size_t)c->p.b * N;
    fast_status st = dalloc_t(c, &sig, nsig ? nsig : 1, s);
    if (!st) {
        c->sig_owned = sig;
        c->sig_owned_bytes = (nsig ? nsig : 1) * 4;
    }
    if (!st) st = dalloc(c, (void **)&d_chunk[0], cbytes, s);
    if (!st) st = dalloc(c, (void **)&d_chunk[1], cbytes, s);
    if (!st) {
        cudaEventRecord(c->chev[2], s);  // the buffers' allocations, ordered on s
        cudaStreamWaitEvent(c->copy_stream, c->chev[2], 0);
        cudaEventRecord(c->chev[3], s);
    }
    // chunk k: filled on the host into staging buffer k % 2 (once that
    // buffer's previous copy is done), copied on the copy stream (once the
    // signature kernel of chunk k - 2 has read the device buffer), signed on s
    for (uint64_t r0 = 0, k = 0; r0 < N && !st; r0 += chunk_rows, k++) {
        const int b = (int)(k & 1);
        const uint64_t n = std::min<uint64_t>(chunk_rows, N - r0);
        if (k >= 2 && (e = cudaEventSynchronize(c->chev[b]))) {
            st = cuda_fail(c, e, "chunk copy");
            break;
        }
        if (fill(user, r0, n, ld, c->h_stage[b]) != 0) {
            st = set_error(c, FAST_EINVAL, "fast_detect_chunked: the fill callback failed at row " + std::to_string(r0));
            break;
        }
        if (k >= 2) cudaStreamWaitEvent(c->copy_stream, c->chev[2 + b], 0);
        cudaMemcpyAsync(d_chunk[b], c->h_stage[b], n * ld * 2, cudaMemcpyHostToDevice, c->copy_stream);
        cudaEventRecord(c->chev[b], c->copy_stream);
        cudaStreamWaitEvent(s, c->chev[b], 0);
        st = sig_launch_rows(c, d_chunk[b], n, ld, sig + r0, N, s);
        cudaEventRecord(c->chev[2 + b], s);
    }
    dfree(c, d_chunk[0], cbytes, s);
    dfree(c, d_chunk[1], cbytes, s);
    stage_mark(c, 1, s);
    if (!st) st = detect_from_sig(c, sig, N, out, s);
    sig_release(c, s);
    if (st) {
        cudaStreamSynchronize(c->copy_stream);  // no copy may still read the staging buffers
        return st;
    }
    stats_times(c, true);
    c->stats.n_fingerprints = N;
    c->stats.peak_bytes = c->peak;
    return FAST_OK;
}

fast_status fast_result_view(const fast_result *r, uint64_t *M, const uint32_t **d_i, const uint32_t **d_j,
                             const uint8_t **d_votes) {
    if (!r) return FAST_EINVAL;
    if (M) *M = r->M;
    if (d_i) *d_i = r->d_i;
    if (d_j) *d_j = r->d_j;
    if (d_votes) *d_votes = r->d_votes;
    return FAST_OK;
}

void fast_result_free(fast_result *r) {
    if (!r) return;
    fast_ctx *c = r->ctx;
    const uint64_t m = r->M ? r->M : 1;
    dfree(c, r->d_i, m * 4, r->stream);
    dfree(c, r->d_j, m * 4, r->stream);
    dfree(c, r->d_votes, m, r->stream);
    delete r;
}

fast_status fast_get_stats(const fast_ctx *c, fast_stats *out) {
    if (!c || !out) return FAST_EINVAL;
    *out = c->stats;
    return FAST_OK;
}

fast_status fast_set_option(fast_ctx *c, const char *name, double value) {
    if (!c || !name) return FAST_EINVAL;
    if (!strcmp(name, "large_min")) c->large_min = (uint32_t)std::max(0.0, value);
    else if (!strcmp(name, "group_pairs")) {
        if (!(value == 0 || (value >= 64 && value <= 8192)))
            return set_error(c, FAST_EINVAL, "group_pairs must be 0 or in [64, 8192]");
        c->group_pairs = (uint32_t)value;
    }
    else if (!strcmp(name, "map_load")) {
        if (!(value > 0.05 && value < 0.95)) return set_error(c, FAST_EINVAL, "map_load must be in (0.05, 0.95)");
        c->map_load = (float)value;
    } else if (!strcmp(name, "timing")) c->timing = value != 0;
    else if (!strcmp(name, "vote_map")) c->vote_map = value != 0;
    else if (!strcmp(name, "single_pass")) c->single_pass = value != 0;
    else if (!strcmp(name, "dense_masks")) c->dense_masks = value != 0;
    else if (!strcmp(name, "group_slots")) {
        if (!(value >= 0 && value <= 65536)) return set_error(c, FAST_EINVAL, "group_slots must be in [0, 65536]");
        c->group_slots = (uint32_t)value;
    }
    else return set_error(c, FAST_EINVAL, std::string("unknown option ") + name);
    return FAST_OK;
}

}  // extern "C"
