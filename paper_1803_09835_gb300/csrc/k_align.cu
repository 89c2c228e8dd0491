// k_align.cu -- the two alignment steps that consume the search's output
// (§7.1, §7.2):
//   channel level  the similarity lists of a station's channels are summed
//                  per pair and thresholded again (§7.1 "Channel Level";
//                  §7.2's sort-merge-reduce: sort by (dt, idx1), merge,
//                  reduce equal entries);
//   station level  entries of the combined list are grouped into thin
//                  diagonal clusters, each reduced to its bounding box, entry
//                  count and summed similarity, small ones pruned (§7.1
//                  "Station Level"; §7.2 "Station").
//
// GB300 design.  Channel level: every channel's (i, j, votes) becomes one
// 64-bit word dt:ib | i:ib | votes:8; one LSD radix sort over the words of
// all channels orders them by (dt, idx1) with equal pairs adjacent; a flag
// pass marks the first entry of each pair whose summed votes reach the
// threshold, a scan places them, a write pass emits (i, j, sum).
// Station level: runs along a diagonal are segments of the (dt, idx1)-ordered
// list cut where dt changes or idx1 jumps by >= gap (flags + scan).  A run
// joins a cluster only from the diagonal just below it, and whether it may
// join depends only on the diagonal on which that cluster started (its
// "origin": the width limit), so the merge is decided run by run in rounds --
// a run decides as soon as the origins of its candidate runs on diagonal
// dt - 1 are known -- instead of one diagonal after another.  Runs on one
// diagonal never influence each other's decision.  Clusters are then summed
// at their root run by atomics, pruned, compacted and ordered by
// (dt_min, idx1_min) with two stable 32-bit radix sorts.
#include <algorithm>
#include <type_traits>

#include "fast_internal.cuh"

struct fast_merged {
    fast_ctx *ctx = nullptr;
    uint64_t M = 0;
    uint32_t *d_i = nullptr;
    uint32_t *d_j = nullptr;
    uint16_t *d_sim = nullptr;
    cudaStream_t stream = nullptr;
};

struct fast_clusters {
    fast_ctx *ctx = nullptr;
    uint64_t n = 0;
    uint64_t *d_box = nullptr;  // [n][6]
    cudaStream_t stream = nullptr;
};

namespace fastgb {
namespace {

constexpr uint32_t kUnknown = 0xFFFFFFFFu;
constexpr uint32_t kNoRun = 0xFFFFFFFFu;

uint32_t width_bits(uint64_t n) {  // bits holding every value below n
    uint32_t b = 1;
    while (b < 64 && (1ull << b) < n) b++;
    return b;
}

unsigned grid_for(const fast_ctx *c, uint64_t n, unsigned threads = 256) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + threads - 1) / threads, (uint64_t)c->num_sms * 8));
}

// --------------------------------------------------------- channel level

// word = dt << (ib + 8) | i << 8 | votes, for entries of one channel
__global__ void k_cm_pack(const uint32_t *__restrict__ I, const uint32_t *__restrict__ J,
                          const uint8_t *__restrict__ V, uint64_t m, uint64_t N, uint32_t ib,
                          unsigned long long *__restrict__ out, uint32_t *err) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = I[k], j = J[k];
        if (j <= i || j >= N) {
            set_err(err, ERR_INPUT);
            out[k] = 0;  // a valid word; the call fails anyway
            continue;
        }
        out[k] = ((unsigned long long)(j - i) << (ib + 8)) | ((unsigned long long)i << 8) | V[k];
    }
}

// keep[k] = 1 iff k is the first entry of its pair and the pair's summed
// votes reach thr
__global__ void k_cm_flag(const unsigned long long *__restrict__ w, uint64_t T, uint32_t thr,
                          uint32_t *__restrict__ keep) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long p = w[k] >> 8;
        uint32_t f = 0;
        if (k == 0 || (w[k - 1] >> 8) != p) {
            uint32_t sum = 0;
            for (uint64_t x = k; x < T && (w[x] >> 8) == p; x++) sum += (uint32_t)(w[x] & 0xFF);
            f = sum >= thr;
        }
        keep[k] = f;
    }
}

__global__ void k_cm_write(const unsigned long long *__restrict__ w, uint64_t T, uint32_t ib,
                           const uint32_t *__restrict__ keep, const uint64_t *__restrict__ pos,
                           uint32_t *__restrict__ oi, uint32_t *__restrict__ oj, uint16_t *__restrict__ os) {
    const unsigned long long imask = (1ull << ib) - 1;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += (uint64_t)gridDim.x * blockDim.x) {
        if (!keep[k]) continue;
        const unsigned long long p = w[k] >> 8;
        uint32_t sum = 0;
        for (uint64_t x = k; x < T && (w[x] >> 8) == p; x++) sum += (uint32_t)(w[x] & 0xFF);
        const uint32_t i = (uint32_t)(p & imask), dt = (uint32_t)(p >> ib);
        const uint64_t o = pos[k];
        oi[o] = i;
        oj[o] = i + dt;
        os[o] = (uint16_t)sum;
    }
}

// --------------------------------------------------------- station level

// head[k] = 1 where a run starts: a new diagonal, or an idx1 step >= gap
__global__ void k_sc_heads(const uint32_t *__restrict__ I, const uint32_t *__restrict__ J, uint64_t n, uint32_t gap,
                           uint32_t *__restrict__ head, uint32_t *err) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = I[k], j = J[k];
        uint32_t h = 1;
        if (j <= i) set_err(err, ERR_INPUT);
        if (k) {
            const uint32_t pi = I[k - 1], pdt = J[k - 1] - pi, dt = j - i;
            if (pdt > dt || (pdt == dt && pi >= i)) set_err(err, ERR_INPUT);  // not in (dt, idx1) order
            h = pdt != dt || i - pi >= gap;
        }
        head[k] = h;
    }
}

struct Runs {
    uint32_t *dt, *s, *e, *n;      // diagonal, first and last idx1, entries
    unsigned long long *sim;       // summed similarity
};

// run of entry k = (heads up to and including k) - 1
__global__ void k_sc_runs(const uint32_t *__restrict__ I, const uint32_t *__restrict__ J,
                          const uint16_t *__restrict__ S, uint64_t n, const uint32_t *__restrict__ head,
                          const uint64_t *__restrict__ hpos, Runs R, uint64_t *__restrict__ start) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = hpos[k] + head[k] - 1;
        const uint32_t i = I[k];
        if (head[k]) {
            R.dt[r] = J[k] - i;
            R.s[r] = i;
            start[r] = k;
        }
        if (k + 1 == n || head[k + 1]) R.e[r] = i;
        atomicAdd(R.sim + r, (unsigned long long)S[k]);
    }
}

__global__ void k_sc_count(const uint32_t *__restrict__ head, const uint64_t *__restrict__ hpos, uint64_t n,
                           const uint64_t *__restrict__ start, uint32_t *__restrict__ rn) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        if (k + 1 == n || head[k + 1]) {
            const uint64_t r = hpos[k] + head[k] - 1;
            rn[r] = (uint32_t)(k + 1 - start[r]);
        }
}

// Candidate runs of run x: the runs of diagonal dt - 1 whose idx1 range comes
// within gap of x's, [c0[x], c1[x]) in run order (on one diagonal the runs
// are disjoint and ascending, so they form one contiguous range).
__global__ void k_sc_cands(Runs R, uint32_t nr, uint32_t gap, uint32_t *__restrict__ c0, uint32_t *__restrict__ c1) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nr; x += gridDim.x * blockDim.x) {
        const uint32_t dt = R.dt[x];
        uint32_t lo = 0, hi = x;  // first run with dt >= dt - 1
        while (lo < hi) {
            const uint32_t m = (lo + hi) / 2;
            if (R.dt[m] + 1 < dt) lo = m + 1;
            else hi = m;
        }
        uint32_t end = lo;  // first run with dt >= dt (at most x)
        {
            uint32_t a = lo, b = x;
            while (a < b) {
                const uint32_t m = (a + b) / 2;
                if (R.dt[m] < dt) a = m + 1;
                else b = m;
            }
            end = a;
        }
        if (lo == end || R.dt[lo] + 1 != dt) {
            c0[x] = c1[x] = 0;
            continue;
        }
        // first y with e_y + gap - 1 >= s_x, then every y with s_y <= e_x + gap - 1
        const uint64_t sx = R.s[x], ex = R.e[x];
        uint32_t a = lo, b = end;
        while (a < b) {
            const uint32_t m = (a + b) / 2;
            if ((uint64_t)R.e[m] + gap - 1 < sx) a = m + 1;
            else b = m;
        }
        uint32_t f = a;
        a = f;
        b = end;
        while (a < b) {
            const uint32_t m = (a + b) / 2;
            if ((uint64_t)R.s[m] <= ex + gap - 1) a = m + 1;
            else b = m;
        }
        c0[x] = f;
        c1[x] = a;
    }
}

// One round of merge decisions: a run joins the first candidate (in idx1
// order) whose cluster started at most width - 1 diagonals below it; it waits
// while a candidate before that one is undecided.
__global__ void k_sc_decide(const uint32_t *__restrict__ dtv, uint32_t nr, uint32_t width,
                            const uint32_t *__restrict__ c0, const uint32_t *__restrict__ c1, uint32_t *origin,
                            uint32_t *__restrict__ parent, unsigned long long *decided) {
    uint32_t mine = 0;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nr; x += gridDim.x * blockDim.x) {
        if (((volatile uint32_t *)origin)[x] != kUnknown) continue;
        const uint32_t dt = dtv[x];
        uint32_t p = kNoRun, o = dt;
        bool ready = true;
        for (uint32_t y = c0[x]; y < c1[x]; y++) {
            const uint32_t oy = ((volatile uint32_t *)origin)[y];
            if (oy == kUnknown) {
                ready = false;
                break;
            }
            if (dt - oy + 1 <= width) {
                p = y;
                o = oy;
                break;
            }
        }
        if (!ready) continue;
        parent[x] = p;
        __threadfence();
        ((volatile uint32_t *)origin)[x] = o;
        mine++;
    }
    if (mine) atomicAdd(decided, (unsigned long long)mine);
}

struct Boxes {
    uint32_t *smin, *emax, *dtmax;
    unsigned long long *n, *sim;
};

__global__ void k_sc_sum(Runs R, uint32_t nr, uint32_t width, const uint32_t *__restrict__ parent, Boxes B,
                         uint32_t *err) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nr; x += gridDim.x * blockDim.x) {
        uint32_t r = x, steps = 0;
        while (parent[r] != kNoRun && steps <= width) {
            r = parent[r];
            steps++;
        }
        if (parent[r] != kNoRun) set_err(err, ERR_INTERNAL);  // a chain longer than the width limit allows
        atomicMin(B.smin + r, R.s[x]);
        atomicMax(B.emax + r, R.e[x]);
        atomicMax(B.dtmax + r, R.dt[x]);
        atomicAdd(B.n + r, (unsigned long long)R.n[x]);
        atomicAdd(B.sim + r, R.sim[x]);
    }
}

__global__ void k_sc_keep(const uint32_t *__restrict__ parent, const unsigned long long *__restrict__ cn, uint32_t nr,
                          uint32_t min_n, uint32_t *__restrict__ keep) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nr; x += gridDim.x * blockDim.x)
        keep[x] = parent[x] == kNoRun && cn[x] >= min_n;
}

// compacted cluster q = root x: its idx1_min (first sort key) and run index
__global__ void k_sc_compact(const uint32_t *__restrict__ keep, const uint64_t *__restrict__ pos, uint32_t nr,
                             const uint32_t *__restrict__ smin, uint32_t *__restrict__ key, uint32_t *__restrict__ root) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nr; x += gridDim.x * blockDim.x)
        if (keep[x]) {
            key[pos[x]] = smin[x];
            root[pos[x]] = x;
        }
}

__global__ void k_sc_gather_dt(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ root, uint64_t nc,
                               const uint32_t *__restrict__ dtv, uint32_t *__restrict__ key, uint32_t *__restrict__ rr) {
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = root[perm[q]];
        key[q] = dtv[x];
        rr[q] = x;
    }
}

__global__ void k_sc_boxes(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ rr, uint64_t nc,
                           const uint32_t *__restrict__ dtv, Boxes B, uint64_t *__restrict__ box) {
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = rr[perm[q]];
        uint64_t *b = box + 6 * q;
        b[0] = dtv[x];
        b[1] = B.dtmax[x];
        b[2] = B.smin[x];
        b[3] = B.emax[x];
        b[4] = B.n[x];
        b[5] = B.sim[x];
    }
}

}  // namespace
}  // namespace fastgb

using namespace fastgb;

extern "C" {

fast_status fast_channel_merge(fast_ctx *c, uint64_t N, uint32_t nch, const uint64_t *h_M, const uint32_t *const *d_i,
                               const uint32_t *const *d_j, const uint8_t *const *d_votes, uint32_t thr,
                               fast_merged **out, void *stream) {
    if (!c || !out) return FAST_EINVAL;
    c->err.clear();
    *out = nullptr;
    if (nch < 1 || nch > 256 || !h_M || !d_i || !d_j || !d_votes)
        return set_error(c, FAST_EINVAL, "fast_channel_merge: 1 to 256 channels with their arrays");
    if (N < 2 || N > (1ull << 28)) return set_error(c, FAST_EINVAL, "fast_channel_merge: N must be in [2, 2^28]");
    uint64_t T = 0;
    for (uint32_t ch = 0; ch < nch; ch++) {
        if (h_M[ch] && (!d_i[ch] || !d_j[ch] || !d_votes[ch]))
            return set_error(c, FAST_EINVAL, "fast_channel_merge: NULL array");
        T += h_M[ch];
    }
    cudaStream_t s = (cudaStream_t)stream;
    c->stats.n_launches = 0;
    const uint32_t ib = width_bits(N);  // i < N and dt < N
    std::vector<std::pair<void *, size_t>> owned;
    auto alloc = [&](auto **ptr, size_t count) -> fast_status {
        using T_ = std::remove_reference_t<decltype(**ptr)>;
        fast_status r = dalloc_t(c, ptr, count ? count : 1, s);
        if (!r) owned.push_back({(void *)*ptr, (count ? count : 1) * sizeof(T_)});
        return r;
    };
    auto release = [&]() {
        for (auto &o : owned) dfree(c, o.first, o.second, s);
        owned.clear();
    };
    fast_merged *res = new fast_merged();
    res->ctx = c;
    res->stream = s;
    unsigned long long *wa = nullptr, *wb = nullptr;
    uint32_t *keep = nullptr;
    uint64_t *pos = nullptr;
    fast_status st;
    if ((st = alloc(&wa, T)) || (st = alloc(&wb, T)) || (st = alloc(&keep, T)) || (st = alloc(&pos, T + 1))) {
        release();
        delete res;
        return st;
    }
    uint64_t off = 0;
    for (uint32_t ch = 0; ch < nch; ch++) {
        if (h_M[ch])
            k_cm_pack<<<grid_for(c, h_M[ch]), 256, 0, s>>>(d_i[ch], d_j[ch], d_votes[ch], h_M[ch], N, ib, wa + off,
                                                           c->d_err), FAST_LAUNCHED(c);
        off += h_M[ch];
    }
    uint64_t *sorted = nullptr;
    st = sort_u64(c, T, reinterpret_cast<uint64_t *>(wa), reinterpret_cast<uint64_t *>(wb), 8, 8 + 2 * ib, &sorted, s);
    const unsigned long long *w = reinterpret_cast<const unsigned long long *>(sorted);
    if (!st && T) {
        k_cm_flag<<<grid_for(c, T), 256, 0, s>>>(w, T, thr, keep), FAST_LAUNCHED(c);
        st = scan_excl(c, keep, pos, T, 1, pos + T, s);
    } else if (!st) {
        cudaMemsetAsync(pos, 0, 8, s);
    }
    if (!st) {
        cudaMemcpyAsync(&res->M, pos + T, 8, cudaMemcpyDeviceToHost, s);
        st = sync_check(c, s, "channel merge");
    }
    const uint64_t m = res->M ? res->M : 1;
    if (!st && !(st = dalloc_t(c, &res->d_i, m, s)) && !(st = dalloc_t(c, &res->d_j, m, s)) &&
        !(st = dalloc_t(c, &res->d_sim, m, s)) && T)
        k_cm_write<<<grid_for(c, T), 256, 0, s>>>(w, T, ib, keep, pos, res->d_i, res->d_j, res->d_sim),
            FAST_LAUNCHED(c);
    release();
    if (!st) st = sync_check(c, s, "channel merge output");
    if (st) {
        fast_merged_free(res);
        return st;
    }
    *out = res;
    return FAST_OK;
}

fast_status fast_merged_view(const fast_merged *r, uint64_t *M, const uint32_t **d_i, const uint32_t **d_j,
                             const uint16_t **d_sim) {
    if (!r) return FAST_EINVAL;
    if (M) *M = r->M;
    if (d_i) *d_i = r->d_i;
    if (d_j) *d_j = r->d_j;
    if (d_sim) *d_sim = r->d_sim;
    return FAST_OK;
}

void fast_merged_free(fast_merged *r) {
    if (!r) return;
    const uint64_t m = r->M ? r->M : 1;
    dfree(r->ctx, r->d_i, m * 4, r->stream);
    dfree(r->ctx, r->d_j, m * 4, r->stream);
    dfree(r->ctx, r->d_sim, m * 2, r->stream);
    delete r;
}

fast_status fast_station_clusters(fast_ctx *c, const uint32_t *d_i, const uint32_t *d_j, const uint16_t *d_sim,
                                  uint64_t n, uint32_t gap, uint32_t width, uint32_t min_n, fast_clusters **out,
                                  void *stream) {
    if (!c || !out) return FAST_EINVAL;
    c->err.clear();
    *out = nullptr;
    if (gap < 1 || width < 1) return set_error(c, FAST_EINVAL, "fast_station_clusters: gap and width must be >= 1");
    if (n && (!d_i || !d_j || !d_sim)) return set_error(c, FAST_EINVAL, "fast_station_clusters: NULL array");
    if (n >= 0xFFFFFFFFull) return set_error(c, FAST_EINVAL, "fast_station_clusters: at most 2^32 - 2 entries");
    cudaStream_t s = (cudaStream_t)stream;
    c->stats.n_launches = 0;
    std::vector<std::pair<void *, size_t>> owned;
    auto alloc = [&](auto **ptr, size_t count) -> fast_status {
        using T_ = std::remove_reference_t<decltype(**ptr)>;
        fast_status r = dalloc_t(c, ptr, count ? count : 1, s);
        if (!r) owned.push_back({(void *)*ptr, (count ? count : 1) * sizeof(T_)});
        return r;
    };
    auto release = [&]() {
        for (auto &o : owned) dfree(c, o.first, o.second, s);
        owned.clear();
    };
    auto fail = [&](fast_status r) {
        release();
        return r;
    };
    fast_clusters *res = new fast_clusters();
    res->ctx = c;
    res->stream = s;
    auto fail_res = [&](fast_status r) {
        release();
        delete res;
        return r;
    };
    if (n == 0) {
        if (fast_status r = dalloc_t(c, &res->d_box, 6, s)) return fail_res(r);
        *out = res;
        return FAST_OK;
    }
    // ---- runs along the diagonals
    uint32_t *head = nullptr;
    uint64_t *hpos = nullptr;
    fast_status st;
    if ((st = alloc(&head, n)) || (st = alloc(&hpos, n + 1))) return fail_res(st);
    k_sc_heads<<<grid_for(c, n), 256, 0, s>>>(d_i, d_j, n, gap, head, c->d_err), FAST_LAUNCHED(c);
    if ((st = scan_excl(c, head, hpos, n, 1, hpos + n, s))) return fail_res(st);
    uint64_t nr64 = 0;
    cudaMemcpyAsync(&nr64, hpos + n, 8, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "station clusters: runs"))) return fail_res(st);
    const uint32_t nr = (uint32_t)nr64;
    Runs R{};
    uint64_t *start = nullptr;
    if ((st = alloc(&R.dt, nr)) || (st = alloc(&R.s, nr)) || (st = alloc(&R.e, nr)) || (st = alloc(&R.n, nr)) ||
        (st = alloc(&R.sim, nr)) || (st = alloc(&start, nr)))
        return fail_res(st);
    cudaMemsetAsync(R.sim, 0, (size_t)nr * 8, s);
    k_sc_runs<<<grid_for(c, n), 256, 0, s>>>(d_i, d_j, d_sim, n, head, hpos, R, start), FAST_LAUNCHED(c);
    k_sc_count<<<grid_for(c, n), 256, 0, s>>>(head, hpos, n, start, R.n), FAST_LAUNCHED(c);
    // ---- candidates on the diagonal below, merge decisions in rounds
    uint32_t *c0 = nullptr, *c1 = nullptr, *origin = nullptr, *parent = nullptr;
    if ((st = alloc(&c0, nr)) || (st = alloc(&c1, nr)) || (st = alloc(&origin, nr)) || (st = alloc(&parent, nr)))
        return fail_res(st);
    k_sc_cands<<<grid_for(c, nr), 256, 0, s>>>(R, nr, gap, c0, c1), FAST_LAUNCHED(c);
    cudaMemsetAsync(origin, 0xFF, (size_t)nr * 4, s);
    unsigned long long *decided = reinterpret_cast<unsigned long long *>(c->d_scal);
    cudaMemsetAsync(decided, 0, 8, s);
    // every round decides at least the undecided run on the lowest diagonal,
    // so nr rounds always suffice; the counter is read every 8 rounds
    uint64_t rounds = 0;
    for (;;) {
        for (int k = 0; k < 8; k++)
            k_sc_decide<<<grid_for(c, nr), 256, 0, s>>>(R.dt, nr, width, c0, c1, origin, parent, decided),
                FAST_LAUNCHED(c);
        rounds += 8;
        cudaMemcpyAsync(c->h_scal, decided, 8, cudaMemcpyDeviceToHost, s);
        if ((st = sync_check(c, s, "station clusters: merge"))) return fail_res(st);
        if (c->h_scal[0] >= nr) break;
        if (rounds > (uint64_t)nr + 8) return fail_res(set_error(c, FAST_EINTERNAL, "cluster merge did not settle"));
    }
    // ---- cluster sums at the roots, pruning, order
    Boxes B{};
    if ((st = alloc(&B.smin, nr)) || (st = alloc(&B.emax, nr)) || (st = alloc(&B.dtmax, nr)) || (st = alloc(&B.n, nr)) ||
        (st = alloc(&B.sim, nr)))
        return fail_res(st);
    cudaMemsetAsync(B.smin, 0xFF, (size_t)nr * 4, s);
    cudaMemsetAsync(B.emax, 0, (size_t)nr * 4, s);
    cudaMemsetAsync(B.dtmax, 0, (size_t)nr * 4, s);
    cudaMemsetAsync(B.n, 0, (size_t)nr * 8, s);
    cudaMemsetAsync(B.sim, 0, (size_t)nr * 8, s);
    k_sc_sum<<<grid_for(c, nr), 256, 0, s>>>(R, nr, width, parent, B, c->d_err), FAST_LAUNCHED(c);
    uint32_t *keep = c0;  // reuse: candidates are no longer needed
    uint64_t *kpos = nullptr;
    if ((st = alloc(&kpos, (uint64_t)nr + 1))) return fail_res(st);
    k_sc_keep<<<grid_for(c, nr), 256, 0, s>>>(parent, B.n, nr, min_n, keep), FAST_LAUNCHED(c);
    if ((st = scan_excl(c, keep, kpos, nr, 1, kpos + nr, s))) return fail_res(st);
    uint64_t nc = 0;
    cudaMemcpyAsync(&nc, kpos + nr, 8, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "station clusters: sums"))) return fail_res(st);
    res->n = nc;
    if ((st = dalloc_t(c, &res->d_box, 6 * (nc ? nc : 1), s))) return fail_res(st);
    if (nc) {
        uint32_t *key = c1, *root = origin;  // reuse
        k_sc_compact<<<grid_for(c, nr), 256, 0, s>>>(keep, kpos, nr, B.smin, key, root), FAST_LAUNCHED(c);
        uint32_t *ka = nullptr, *va = nullptr, *kb = nullptr, *vb = nullptr, *key2 = nullptr, *rr = nullptr;
        if ((st = alloc(&ka, nc)) || (st = alloc(&va, nc)) || (st = alloc(&kb, nc)) || (st = alloc(&vb, nc)) ||
            (st = alloc(&key2, nc)) || (st = alloc(&rr, nc))) {
            fast_clusters_free(res);
            return fail(st);
        }
        uint32_t *k1 = nullptr, *p1 = nullptr, *k2 = nullptr, *p2 = nullptr;
        // idx1_min first, then a stable pass on dt_min: (dt_min, idx1_min) order
        st = sort_u32(c, 1, nc, key, nullptr, ka, va, kb, vb, 0, 32, &k1, &p1, s, nullptr);
        if (!st) {
            k_sc_gather_dt<<<grid_for(c, nc), 256, 0, s>>>(p1, root, nc, R.dt, key2, rr), FAST_LAUNCHED(c);
            uint32_t *pa = p1 == va ? vb : va;  // scratch not holding p1
            uint32_t *ka2 = p1 == va ? kb : ka;
            // rr is indexed by the first order's position: sort the positions
            st = sort_u32(c, 1, nc, key2, nullptr, ka2, pa, key, parent, 0, 32, &k2, &p2, s, nullptr);
        }
        if (!st)
            k_sc_boxes<<<grid_for(c, nc), 256, 0, s>>>(p2, rr, nc, R.dt, B, res->d_box), FAST_LAUNCHED(c);
    }
    release();
    if (!st) st = sync_check(c, s, "station clusters");
    if (st) {
        fast_clusters_free(res);
        return st;
    }
    *out = res;
    return FAST_OK;
}

fast_status fast_clusters_view(const fast_clusters *r, uint64_t *n, const uint64_t **d_box) {
    if (!r) return FAST_EINVAL;
    if (n) *n = r->n;
    if (d_box) *d_box = r->d_box;
    return FAST_OK;
}

void fast_clusters_free(fast_clusters *r) {
    if (!r) return;
    dfree(r->ctx, r->d_box, 6 * 8 * (r->n ? r->n : 1), r->stream);
    delete r;
}

}  // extern "C"
