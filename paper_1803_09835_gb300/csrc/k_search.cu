// k_search.cu -- occurrence filter (§6.5), pair enumeration inside buckets and
// vote counting (§6.1 "Search", §6.3), threshold and canonical output (§7.2).
//
// votes(i, j) = number of tables in which i and j share a bucket; a pair is
// reported when neither is dropped, j - i > excl and votes >= v.
//
// GB300 design.  Every bucket pair is one "emission"; emissions from all b
// tables must be summed per pair.  Buckets come in two very different kinds:
//   * sparse: the background, sizes ~2..50, almost every pair seen once.
//     Default (row-partitioned) path: one pass over the tables appends every
//     pair (i, j), as a packed (row-in-group, j) word, to the region of its
//     row group (2^gshift consecutive ids i; a fixed number of slots per group,
//     the rare excess in an overflow list); a warp per group then counts the
//     votes of its pairs in shared memory (a counting filter first, an exact
//     hash for the few that pass) and keeps those with votes >= v in (i, j)
//     order.  When the regions do not fit, a counting pass sizes the groups
//     exactly and a writing pass fills them.  The rows are assembled into the
//     canonical list with one scan, no global sort.  Alternative path
//     (`vote_map`): one device open-addressing map of packed (i, j) -> votes
//     (a 64-bit slot: i:28 | j:28 | votes:8) per query partition, then a radix
//     sort of the kept pairs.
//   * dense: a repeating source (e.g. periodic noise) puts thousands of
//     near-copies in one bucket in most tables, so the same pairs recur in
//     every table -- ~10^10 emissions for ~10^8 distinct pairs.  Buckets with
//     at least `large_min` live members (and at least 1/16 of the largest
//     bucket's) are merged into groups (connected components of shared large
//     buckets); for every pair inside a group the votes are computed once per
//     pair instead of once per table: from bit masks of the group's large
//     same-key clusters (popcount) plus the pairs of its small clusters, or,
//     for a group with too many large clusters, by comparing the two
//     fingerprints' b keys tile by tile in shared memory.  The sparse path
//     skips pairs inside a group, so each pair is counted by exactly one of
//     the two paths, and both count exactly the definition.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <type_traits>

#include "fast_internal.cuh"

namespace fastgb {

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kSmall = 32;  // buckets up to this size are enumerated by one thread

// -------------------------------------------------------------- filter

// Heavy bucket starts by a scan of the keys, for thresholds within the small
// bucket sizes: size >= smin, i.e. occ_den * size > occ_num * N_s, N_s the size
// of the bucket's station.
__global__ void k_heavy_find(const uint32_t *__restrict__ skey, uint64_t N, Stations S, uint32_t occ_num,
                             uint32_t occ_den, uint4 *__restrict__ list, unsigned long long *__restrict__ count,
                             uint64_t cap, uint32_t *err) {
    const uint32_t t = blockIdx.y;
    const uint32_t *k = skey + (uint64_t)t * N;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t sx = station_of(S, p);
        const uint64_t s0 = S.soff[sx], s1 = S.soff[sx + 1];
        const uint64_t smin = (uint64_t)occ_num * (s1 - s0) / occ_den + 1;
        const uint32_t key = k[p];
        if (p > s0 && k[p - 1] == key) continue;
        if (p + smin - 1 >= s1 || k[p + smin - 1] != key) continue;
        // gallop then bisect to the end of the run
        uint64_t lo = p + smin - 1, step = 1, hi;
        for (;;) {
            hi = lo + step;
            if (hi >= s1 || k[hi] != key) break;
            lo = hi;
            step <<= 1;
        }
        if (hi > s1) hi = s1;
        while (hi - lo > 1) {  // k[lo] == key, k[hi] != key or hi == s1
            uint64_t mid = lo + (hi - lo) / 2;
            if (k[mid] == key) lo = mid;
            else hi = mid;
        }
        unsigned long long slot = atomicAdd(count, 1ull);
        if (slot < cap) list[slot] = make_uint4(t, (uint32_t)p, (uint32_t)hi, 0);
        else set_err(err, ERR_OVERFLOW);
    }
}

// Heavy buckets, from the list of big ones: occ_den * size > occ_num * N_s
// (N_s the size of the bucket's station); every id in a heavy bucket counts
// one more table.
__global__ void k_heavy_mark_list(const uint4 *__restrict__ list, const unsigned long long *__restrict__ count,
                                  uint64_t cap, const uint32_t *__restrict__ sid, uint64_t N, uint32_t *__restrict__ heavy) {
    const uint64_t n = min((uint64_t)*count, cap);
    for (uint64_t b = blockIdx.x; b < n; b += gridDim.x) {
        uint4 e = list[b];
        const uint32_t *s = sid + (uint64_t)e.x * N;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) atomicAdd(&heavy[s[q]], 1u);
    }
}

__global__ void k_heavy_mark(const uint4 *__restrict__ big, const unsigned long long *__restrict__ count,
                             uint64_t cap, Stations S, uint32_t occ_num, uint32_t occ_den,
                             const uint32_t *__restrict__ sid, uint64_t N, uint32_t *__restrict__ heavy) {
    const uint64_t n = min((uint64_t)*count, cap);
    for (uint64_t bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const uint4 e = big[bi];
        const uint32_t sx = station_of(S, e.y);
        const uint64_t ns = S.soff[sx + 1] - S.soff[sx];
        if ((uint64_t)occ_den * (e.z - e.y) <= (uint64_t)occ_num * ns) continue;  // block-uniform
        const uint32_t *s = sid + (uint64_t)e.x * N;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) atomicAdd(&heavy[s[q]], 1u);
    }
}

__global__ void k_drop(const uint32_t *__restrict__ heavy, uint64_t N, uint32_t nb, uint8_t *__restrict__ drop,
                       unsigned long long *__restrict__ ndrop) {
    uint32_t mine = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t d = heavy ? (uint8_t)(2ull * heavy[i] > nb) : 0;
        drop[i] = d;
        mine += d;
    }
    for (int o = 16; o; o >>= 1) mine += __shfl_down_sync(~0u, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(ndrop, (unsigned long long)mine);
}

// ---------------------------------------------------------- vote map

// --------------------------------------------------- bucket enumeration

struct EnumArgs {
    const uint32_t *skey, *sid;
    const uint8_t *drop;
    const uint32_t *label;  // nullptr before grouping
    const uint32_t *fsid;   // sid with bit 31 set on dropped ids and group members (nullptr: not built)
    uint64_t N;
    uint32_t excl;
    uint32_t i_lo, i_hi;  // query partition [i_lo, i_hi)
    uint32_t nparts;      // counting: partition of i is i * nparts / N
    Stations st;          // station ranges: buckets never cross them
    const uint32_t *fbits;  // flag bitmap over ids (dropped or in a dense group); with fsid_out:
    uint32_t *fsid_out;     // the counting pass writes fsid while it reads sid
};

__device__ __forceinline__ bool pair_live(const EnumArgs &a, uint32_t i, uint32_t j) {
    if (j - i <= a.excl) return false;
    if (a.label) {
        uint32_t li = __ldg(a.label + i);
        if (li != kNone && li == __ldg(a.label + j)) return false;
    }
    return true;
}

// mode 0: find big buckets (size > kSmall) and count small-bucket pairs per
//         query partition (an upper bound: group membership is not known yet)
// mode 1: add small-bucket pairs with i in [i_lo, i_hi) to the vote map
template <int MODE>
__global__ void __launch_bounds__(256) k_enum(EnumArgs a, uint4 *__restrict__ big, unsigned long long *__restrict__ nbig,
                                              uint64_t big_cap, unsigned long long *__restrict__ part_cnt, Map map,
                                              uint32_t *err) {
    __shared__ unsigned long long s_cnt[64];
    if (MODE == 0) {
        for (int i = threadIdx.x; i < 64; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
    }
    const uint32_t t = blockIdx.y;
    const uint64_t N = a.N;
    const uint32_t *k = a.skey + (uint64_t)t * N;
    const uint32_t *s = a.sid + (uint64_t)t * N;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t sx = station_of(a.st, p);
        const uint64_t s0 = a.st.soff[sx], s1 = a.st.soff[sx + 1];
        const uint32_t key = k[p];
        if (p > s0 && k[p - 1] == key) continue;
        uint64_t e = p + 1;
        while (e < s1 && e - p <= kSmall && k[e] == key) e++;
        if (e - p == 1) continue;
        if (e - p > kSmall) {
            if (MODE == 0) {
                uint64_t lo = e - 1, step = 1, hi;
                for (;;) {
                    hi = lo + step;
                    if (hi >= s1 || k[hi] != key) break;
                    lo = hi;
                    step <<= 1;
                }
                if (hi > s1) hi = s1;
                while (hi - lo > 1) {
                    uint64_t mid = lo + (hi - lo) / 2;
                    if (k[mid] == key) lo = mid;
                    else hi = mid;
                }
                unsigned long long slot = atomicAdd(nbig, 1ull);
                if (slot < big_cap) big[slot] = make_uint4(t, (uint32_t)p, (uint32_t)hi, 0);
                else set_err(err, ERR_OVERFLOW);
            }
            continue;
        }
        for (uint64_t x = p; x < e; x++) {
            const uint32_t i = s[x];
            if (a.drop[i]) continue;
            if (MODE == 1 && (i < a.i_lo || i >= a.i_hi)) continue;
            uint32_t c = 0;
            for (uint64_t y = x + 1; y < e; y++) {
                const uint32_t j = s[y];
                if (a.drop[j] || !pair_live(a, i, j)) continue;
                if (MODE == 1) map_add(map, pair_key(i, j), err);
                else ++c;
            }
            if (MODE == 0 && c) atomicAdd(&s_cnt[(uint64_t)i * a.nparts / N], (unsigned long long)c);
        }
    }
    if (MODE == 0) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < a.nparts; i += blockDim.x)
            if (s_cnt[i]) atomicAdd(part_cnt + i, s_cnt[i]);
    }
}

// Block-wide exclusive scan helper for 0/1 flags (blockDim multiple of 32, <= 1024).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *wsum, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(~0u, v, d);
        if (lane >= d) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(~0u, w, d);
            if (lane >= d) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t r = v - x + (warp ? wsum[warp - 1] : 0);
    *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

// Classifies big buckets by live size: >= large_min -> large list (dense
// path), otherwise medium list; counts medium pairs per query partition
// (each live member i pairs with the live members after it).  With lm_st,
// a batch's station x has threshold lm_st[x] and its largest live bucket
// goes to lmax_st[x].
__global__ void __launch_bounds__(256) k_big_classify(EnumArgs a, uint4 *__restrict__ big,
                                                      const unsigned long long *__restrict__ nbig, uint64_t big_cap,
                                                      uint32_t large_min, uint4 *__restrict__ large,
                                                      unsigned long long *__restrict__ nlarge, uint4 *__restrict__ medium,
                                                      unsigned long long *__restrict__ nmedium,
                                                      unsigned long long *__restrict__ part_cnt,
                                                      unsigned long long *__restrict__ lmax = nullptr,
                                                      const uint32_t *__restrict__ lm_st = nullptr,
                                                      unsigned long long *__restrict__ lmax_st = nullptr) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_live;
    __shared__ unsigned long long s_cnt[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) s_cnt[i] = 0;
    const uint64_t n = min((uint64_t)*nbig, big_cap);
    for (uint64_t bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const uint4 e = big[bi];
        const uint32_t *s = a.sid + (uint64_t)e.x * a.N;
        // live members: counted once per table set and kept in the entry's w
        // (live + 1; 0 = not counted yet): they depend only on the drop mask
        uint32_t nl;
        if (e.w) {  // block-uniform
            nl = e.w - 1;
        } else {
            uint32_t live = 0;
            for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) live += !a.drop[s[q]];
            for (int o = 16; o; o >>= 1) live += __shfl_down_sync(~0u, live, o);
            if (threadIdx.x == 0) s_live = 0;
            __syncthreads();
            if ((threadIdx.x & 31) == 0) atomicAdd(&s_live, live);
            __syncthreads();
            nl = s_live;
            if (threadIdx.x == 0) big[bi].w = nl + 1;
        }
        uint32_t large_min_b = large_min;
        if (lm_st) {  // block-uniform
            const uint32_t x = station_of(a.st, e.y);
            large_min_b = lm_st[x];
            if (threadIdx.x == 0 && lmax_st) atomicMax(lmax_st + x, (unsigned long long)nl);
        }
        if (threadIdx.x == 0 && lmax) atomicMax(lmax, (unsigned long long)nl);
        if (threadIdx.x == 0 && nl >= 2) {
            if (nl >= large_min_b) large[atomicAdd(nlarge, 1ull)] = make_uint4(e.x, e.y, e.z, nl);
            else medium[atomicAdd(nmedium, 1ull)] = make_uint4(e.x, e.y, e.z, nl);
        }
        if (a.nparts == 1) {  // one partition: the bucket's pairs are C(nl, 2)
            if (threadIdx.x == 0 && nl >= 2 && nl < large_min_b) s_cnt[0] += (unsigned long long)nl * (nl - 1) / 2;
        } else if (nl >= 2 && nl < large_min_b) {
            uint32_t rank0 = 0;
            for (uint32_t q0 = e.y; q0 < e.z; q0 += blockDim.x) {
                const uint32_t q = q0 + threadIdx.x;
                uint32_t id = 0, lv = 0;
                if (q < e.z) {
                    id = s[q];
                    lv = !a.drop[id];
                }
                uint32_t tot;
                const uint32_t r = rank0 + block_excl_scan(lv, wsum, &tot);
                if (lv && nl - 1 - r) atomicAdd(&s_cnt[(uint64_t)id * a.nparts / a.N], (unsigned long long)(nl - 1 - r));
                rank0 += tot;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < a.nparts; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(part_cnt + i, s_cnt[i]);
}

// Adds the pairs of medium buckets (live size < large_min) to the vote map.
// One CTA per bucket.  Buckets with at most kMedSmem live members are
// compacted into shared memory first; larger ones are read in place.
constexpr uint32_t kMedSmem = 8192;

__global__ void __launch_bounds__(256) k_medium(EnumArgs a, const uint4 *__restrict__ medium,
                                                const unsigned long long *__restrict__ nmedium, Map map, uint32_t *err) {
    __shared__ uint32_t s_m[kMedSmem];
    __shared__ uint32_t wsum[32];
    const uint64_t n = *nmedium;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint64_t bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const uint4 e = medium[bi];
        const uint32_t *s = a.sid + (uint64_t)e.x * a.N;
        if (e.w <= kMedSmem) {
            uint32_t nl = 0;
            for (uint32_t q0 = e.y; q0 < e.z; q0 += blockDim.x) {
                const uint32_t q = q0 + threadIdx.x;
                uint32_t id = 0, live = 0;
                if (q < e.z) {
                    id = s[q];
                    live = !a.drop[id];
                }
                uint32_t tot;
                const uint32_t pos = block_excl_scan(live, wsum, &tot);
                if (live && nl + pos < kMedSmem) s_m[nl + pos] = id;
                nl += tot;
            }
            nl = min(nl, kMedSmem);
            __syncthreads();
            for (uint32_t x = warp; x < nl; x += nw) {
                const uint32_t i = s_m[x];
                if (i < a.i_lo || i >= a.i_hi) continue;
                for (uint32_t y = x + 1 + lane; y < nl; y += 32) {
                    const uint32_t j = s_m[y];
                    if (pair_live(a, i, j)) map_add(map, pair_key(i, j), err);
                }
            }
        } else {
            for (uint32_t x = e.y + warp; x < e.z; x += nw) {
                const uint32_t i = s[x];
                if (a.drop[i] || i < a.i_lo || i >= a.i_hi) continue;
                for (uint32_t y = x + 1 + lane; y < e.z; y += 32) {
                    const uint32_t j = s[y];
                    if (!a.drop[j] && pair_live(a, i, j)) map_add(map, pair_key(i, j), err);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ grouping

__global__ void k_label_init(const uint4 *__restrict__ large, uint64_t nlarge, const uint32_t *__restrict__ sid,
                             const uint8_t *__restrict__ drop, uint64_t N, uint32_t *__restrict__ label) {
    __shared__ uint32_t s_min;
    for (uint64_t bi = blockIdx.x; bi < nlarge; bi += gridDim.x) {
        const uint4 e = large[bi];
        const uint32_t *s = sid + (uint64_t)e.x * N;
        if (threadIdx.x == 0) s_min = kNone;
        __syncthreads();
        uint32_t mn = kNone;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) {
            uint32_t id = s[q];
            if (!drop[id]) mn = min(mn, id);
        }
        atomicMin(&s_min, mn);
        __syncthreads();
        mn = s_min;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) {
            uint32_t id = s[q];
            if (!drop[id]) atomicMin(&label[id], mn);
        }
        __syncthreads();
    }
}

// One round of min-label propagation over large buckets, plus pointer jumping.
__global__ void k_label_prop(const uint4 *__restrict__ large, uint64_t nlarge, const uint32_t *__restrict__ sid,
                             const uint8_t *__restrict__ drop, uint64_t N, uint32_t *__restrict__ label,
                             uint32_t *__restrict__ changed) {
    __shared__ uint32_t s_min;
    for (uint64_t bi = blockIdx.x; bi < nlarge; bi += gridDim.x) {
        const uint4 e = large[bi];
        const uint32_t *s = sid + (uint64_t)e.x * N;
        if (threadIdx.x == 0) s_min = kNone;
        __syncthreads();
        uint32_t mn = kNone;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) {
            uint32_t id = s[q];
            if (!drop[id]) {
                uint32_t l = __ldcg(label + id);
                uint32_t ll = __ldcg(label + l);  // label of the label (pointer jumping)
                mn = min(mn, min(l, ll));
            }
        }
        atomicMin(&s_min, mn);
        __syncthreads();
        mn = s_min;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) {
            uint32_t id = s[q];
            if (!drop[id]) {
                uint32_t old = atomicMin(&label[id], mn);
                if (old > mn) *changed = 1;
            }
        }
        __syncthreads();
    }
}

__global__ void k_collect_members(const uint32_t *__restrict__ label, uint64_t N,
                                  unsigned long long *__restrict__ memb, unsigned long long *__restrict__ cnt) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l = label[i];
        if (l != kNone) memb[atomicAdd(cnt, 1ull)] = ((unsigned long long)l << 32) | i;
    }
}

// GT[t][k] = key of member k in table t (members compacted, table-major).
__global__ void k_gather_keys(const unsigned long long *__restrict__ memb, uint64_t nm, const uint32_t *__restrict__ sig,
                              uint64_t N, uint32_t nb, uint32_t *__restrict__ GT, uint32_t *__restrict__ ids) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nm; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t id = (uint32_t)memb[k];
        ids[k] = id;
        for (uint32_t t = 0; t < nb; t++) GT[(uint64_t)t * nm + k] = __ldg(sig + (uint64_t)t * N + id);
    }
}

// ------------------------------------------------------------ dense tiles

constexpr int kDT = 64;  // tile edge

struct DenseTile {
    uint32_t g0;   // first member of the group
    uint32_t n;    // group size
    uint32_t ta, tb;
};

// Direct votes of every pair inside a tile of one group.  MODE 0 counts the
// detections, MODE 1 writes them (packed for the final sort).
template <int MODE>
__global__ void __launch_bounds__(256) k_dense(const DenseTile *__restrict__ tiles, uint64_t ntiles,
                                               const uint32_t *__restrict__ GT, const uint32_t *__restrict__ ids,
                                               uint64_t nm, uint32_t nb, uint32_t v, uint32_t excl, uint32_t nbits,
                                               unsigned long long *__restrict__ out, unsigned long long *__restrict__ cursor,
                                               uint64_t cap, uint32_t *err) {
    extern __shared__ uint32_t sd[];
    uint32_t *sA = sd;                    // [nb][64]
    uint32_t *sB = sd + (size_t)nb * kDT;  // [nb][64]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int lane = threadIdx.x & 31;
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const DenseTile T = tiles[ti];
        const uint32_t a0 = T.g0 + T.ta * kDT, b0 = T.g0 + T.tb * kDT;
        const uint32_t na = min((uint32_t)kDT, T.n - T.ta * kDT), nbb = min((uint32_t)kDT, T.n - T.tb * kDT);
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < nb * kDT; x += blockDim.x) {
            const uint32_t t = x / kDT, c = x % kDT;
            sA[x] = c < na ? GT[(uint64_t)t * nm + a0 + c] : 0xFFFFFFFFu;
            sB[x] = c < nbb ? GT[(uint64_t)t * nm + b0 + c] : 0xFFFFFFFEu;
        }
        __syncthreads();
        uint32_t acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int w = 0; w < 4; w++) acc[u][w] = 0;
        for (uint32_t t = 0; t < nb; t++) {
            const uint4 av = *reinterpret_cast<const uint4 *>(sA + t * kDT + ty * 4);
            const uint4 bv = *reinterpret_cast<const uint4 *>(sB + t * kDT + tx * 4);
            const uint32_t A[4] = {av.x, av.y, av.z, av.w}, B[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int w = 0; w < 4; w++) acc[u][w] += A[u] == B[w];
        }
        uint32_t cnt = 0;
        unsigned long long pk[16];
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const uint32_t ga = T.ta * kDT + ty * 4 + u, gb = T.tb * kDT + tx * 4 + w;
                pk[u * 4 + w] = 0;
                if (ga < T.n && gb < T.n && ga < gb && acc[u][w] >= v) {
                    const uint32_t i = ids[T.g0 + ga], j = ids[T.g0 + gb];
                    if (j - i > excl) {
                        pk[u * 4 + w] = ((unsigned long long)i << (nbits + 8)) | ((unsigned long long)j << 8) | acc[u][w];
                        ++cnt;
                    }
                }
            }
        // warp-aggregated reservation
        uint32_t pre = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(~0u, pre, d);
            if (lane >= d) pre += y;
        }
        const uint32_t wtot = __shfl_sync(~0u, pre, 31);
        unsigned long long base = 0;
        if (lane == 31 && wtot) base = atomicAdd(cursor, (unsigned long long)wtot);
        base = __shfl_sync(~0u, base, 31);
        if (MODE == 1 && cnt) {
            unsigned long long o = base + pre - cnt;
#pragma unroll
            for (int x = 0; x < 16; x++)
                if (pk[x]) {
                    if (o < cap) out[o] = pk[x];
                    else set_err(err, ERR_OVERFLOW);
                    ++o;
                }
        }
    }
}

// --------------------------------------------------------- map output

template <int MODE>
__global__ void k_map_compact(const unsigned long long *__restrict__ slot, uint64_t cap, uint32_t v, uint32_t nbits,
                              unsigned long long *__restrict__ out, unsigned long long *__restrict__ cursor,
                              uint64_t out_cap, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_iter = (cap + stride - 1) / stride;
    for (uint64_t it = 0; it < n_iter; it++) {
        const uint64_t s = it * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        unsigned long long val = s < cap ? __ldcs(slot + s) : 0ull;
        const bool keep = val != 0 && (uint32_t)(val & 0xFF) >= v;
        const uint32_t ballot = __ballot_sync(~0u, keep);
        if (!ballot) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)__popc(ballot));
        base = __shfl_sync(~0u, base, 0);
        if (MODE == 1 && keep) {
            const uint64_t key = val >> 8;
            const uint64_t i = key >> 28, j = key & ((1u << 28) - 1);
            const unsigned long long o = base + __popc(ballot & ((1u << lane) - 1));
            if (o < out_cap) out[o] = (i << (nbits + 8)) | (j << 8) | (val & 0xFF);
            else set_err(err, ERR_OVERFLOW);
        }
    }
}

__global__ void k_unpack(const unsigned long long *__restrict__ in, uint64_t M, uint32_t nbits, uint32_t *__restrict__ oi,
                         uint32_t *__restrict__ oj, uint8_t *__restrict__ ov) {
    const uint64_t jm = (1ull << nbits) - 1;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = in[x];
        oi[x] = (uint32_t)(k >> (nbits + 8));
        oj[x] = (uint32_t)((k >> 8) & jm);
        ov[x] = (uint8_t)(k & 0xFF);
    }
}

// ------------------------------------------------- row-partitioned votes

__device__ __forceinline__ uint32_t row_hash(uint32_t j) { return (uint32_t)(mix64(j) >> 32); }

// Kept entries of one row, written in j order: each kept entry's rank is the
// number of kept entries with a smaller j (j is unique within a row).
__device__ __forceinline__ void row_write_sorted(const uint32_t *kj, const uint32_t *kv, uint32_t nk, uint32_t lane,
                                                 uint32_t nlanes, uint32_t *sp_j, uint8_t *sp_v, uint64_t base) {
    for (uint32_t x = lane; x < nk; x += nlanes) {
        const uint32_t jx = kj[x];
        uint32_t rank = 0;
        for (uint32_t y = 0; y < nk; y++) rank += kj[y] < jx;
        sp_j[base + rank] = jx;
        sp_v[base + rank] = (uint8_t)kv[x];
    }
}

constexpr uint32_t kRowBlockSlots = 16384;  // shared-memory hash of the one-CTA-per-row path

// ------------------------------------------------- group-partitioned votes
//
// Rows (pairs keyed by their lower id i) are cut into groups of 2^gshift
// consecutive ids.  Bucket-major passes over the sorted tables count each
// group's pairs, then append every pair to its group's region as one packed
// entry (i's offset in the group, j); with one open sector per group the
// write frontier stays in L2.  A CTA per group then sorts its entries by row
// in shared memory and counts each row's duplicates of j in a hash: the
// number of tables in which i and j share a bucket (§6.1 "Search").

template <typename PT>
__device__ __forceinline__ PT pack_entry(uint32_t local, uint32_t j, uint32_t nbits) {
    return ((PT)local << nbits) | (PT)j;
}

// Small buckets (at most kSmall entries, dropped ones included).  A warp walks
// a run of 32-entry tiles of one table with a window of three tiles in
// registers -- previous (bucket heads only), current and next -- so every key,
// id, drop flag and group label is loaded once.  Lane L owns position L of the
// current tile and pairs it with the later entries of its bucket, which lie in
// the current or the next tile (a small bucket spans at most 32 positions);
// their ids and labels come by shuffle.  Bucket bounds come from the head
// bitmasks: a head is a position whose key differs from its predecessor's, or
// the first position of a station.
constexpr uint32_t kLabDrop = 0xFFFFFFFEu;  // window label of a dropped (or absent) entry

struct PairWin {
    uint32_t id, lab, heads, key;
};

// kprev0: the key at position 32 T - 1 (the previous tile's last), unused for T = 0.
__device__ __forceinline__ PairWin pair_tile(const EnumArgs &a, const uint32_t *__restrict__ K,
                                             const uint32_t *__restrict__ S, const uint32_t *__restrict__ FS,
                                             uint32_t *__restrict__ FO, uint64_t T, bool own, uint32_t kprev0) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t x = T * 32 + lane, N = a.N;
    const bool valid = x < N;
    const uint32_t key = valid ? __ldcs(K + x) : 0u;
    uint32_t kprev = __shfl_up_sync(~0u, key, 1);
    if (lane == 0) kprev = kprev0;
    bool head = !valid || x == 0 || key != kprev;
    if (a.st.nst > 1 && valid && !head) head = a.st.soff[station_of(a.st, x)] == x;
    PairWin w;
    w.key = key;
    w.heads = __ballot_sync(~0u, head);
    w.lab = kLabDrop;
    if (FS || a.fbits) {  // only flagged entries (dropped or in a dense group) need the random lookups
        uint32_t raw = 0;
        if (FS) {
            raw = valid ? __ldcs(FS + x) : 0u;
        } else if (valid) {  // flag the id from the bitmap (the counting pass keeps the flagged copy)
            const uint32_t id = __ldcs(S + x);
            raw = id | (__ldg(a.fbits + (id >> 5)) >> (id & 31)) << 31;
            if (own && FO) FO[x] = raw;
        }
        w.id = raw & 0x7FFFFFFFu;
        if (valid) w.lab = !(raw >> 31) ? kNone : a.drop[w.id] ? kLabDrop : __ldg(a.label + w.id);
    } else {
        w.id = valid ? S[x] : 0u;
        if (valid && !a.drop[w.id]) w.lab = a.label ? __ldg(a.label + w.id) : kNone;
    }
    return w;
}

// Flag bitmap over ids: bit id set iff id is dropped or a dense-group member.
__global__ void __launch_bounds__(256) k_flag_bits(const uint8_t *__restrict__ drop, const uint32_t *__restrict__ label,
                                                   uint64_t N, uint32_t *__restrict__ bits) {
    const uint64_t nw = (N + 31) / 32;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0;
        for (uint32_t k = 0; k < 32; k++) {
            const uint64_t id = w * 32 + k;
            if (id < N && (drop[id] || label[id] != kNone)) m |= 1u << k;
        }
        bits[w] = m;
    }
}



// Row groups [g_lo, g_hi) written by one emission pass; their entries start at
// goff[g] - ebase in that pass's buffer (all groups, ebase 0, when unsplit).
struct GroupRange {
    uint64_t g_lo, g_hi, ebase;
    __device__ __forceinline__ bool has(uint64_t g) const { return g >= g_lo && g < g_hi; }
};

// Single-pass emission (MODE 2): every row group owns `cap` slots of `region`;
// entries past them go to an overflow list of (group, entry), placed after
// the region's entries when the groups are compacted to exact offsets.
struct RegionSink {
    uint32_t *region;
    uint32_t cap;
    unsigned long long *ovf, ovf_cap, *novf;
    __device__ __forceinline__ void put(uint64_t g, uint64_t slot, uint32_t e) const {
        if (slot < cap) {
            region[g * cap + slot] = e;
        } else {
            const unsigned long long q = atomicAdd(novf, 1ull);
            if (q < ovf_cap) ovf[q] = (unsigned long long)g << 32 | e;
        }
    }
};

// Slots for cnt new pairs of row group g: the single pass counts from 0 in
// gcur (its regions are fixed); the counted pass takes them from the
// group's cursor gpos, which starts at the group's offset in the pass's
// buffer (one atomic, no offset lookup).
template <int MODE>
__device__ __forceinline__ uint64_t reserve(uint32_t *gcur, unsigned long long *gpos, uint64_t g, uint32_t cnt) {
    if (MODE == 2) return atomicAdd(gcur + g, cnt);
    return atomicAdd(gpos + g, (unsigned long long)cnt);
}

// gpos[g] = goff[g] - ebase for the groups of one pass.
__global__ void k_init_pos(const uint64_t *__restrict__ goff, GroupRange gr, unsigned long long *__restrict__ gpos) {
    for (uint64_t g = gr.g_lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < gr.g_hi;
         g += (uint64_t)gridDim.x * blockDim.x)
        gpos[g] = goff[g] - gr.ebase;
}

struct PairSmem {  // one warp's tile window and its pair bookkeeping
    uint32_t id[64], lab[64], pre[32];
    uint64_t keep[32];  // per row: window positions of its kept partners
    uint64_t base[32];
};

template <int MODE, typename PT>
__global__ void __launch_bounds__(256) k_pairs_grp(EnumArgs a, uint32_t gshift, uint32_t nbits, uint32_t tiles_per_warp,
                                                   uint32_t *__restrict__ gcnt, unsigned long long *__restrict__ gpos,
                                                   uint32_t *__restrict__ gcur, PT *__restrict__ ent,
                                                   unsigned long long *__restrict__ n_emit, GroupRange gr,
                                                   RegionSink rs = RegionSink{}) {
    const uint32_t t = blockIdx.y, lane = threadIdx.x & 31;
    const uint64_t N = a.N, ntiles = (N + 31) / 32;
    const uint32_t *K = a.skey + (uint64_t)t * N;
    const uint32_t *S = a.sid + (uint64_t)t * N;
    const uint32_t *FS = MODE == 1 && a.fsid ? a.fsid + (uint64_t)t * N : nullptr;
    uint32_t *FO = MODE == 0 && a.fsid_out ? a.fsid_out + (uint64_t)t * N : nullptr;
    const uint32_t lmask = (1u << gshift) - 1;
    const uint64_t T0 = ((uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * tiles_per_warp;
    if (T0 >= ntiles) return;  // warp-uniform
    const uint64_t T1 = min(T0 + tiles_per_warp, ntiles);
    __shared__ PairSmem ps[8];
    PairSmem &W = ps[threadIdx.x / 32];
    uint32_t hp = ~0u, kp0 = 0;
    if (T0) {
        const PairWin pw = pair_tile(a, K, S, FS, FO, T0 - 1, false, T0 > 1 ? K[(T0 - 1) * 32 - 1] : 0u);
        hp = pw.heads;
        kp0 = __shfl_sync(~0u, pw.key, 31);
    }
    PairWin c = pair_tile(a, K, S, FS, FO, T0, true, kp0);
    unsigned long long emitted = 0;  // counting pass: pairs of this lane's entries
    for (uint64_t T = T0; T < T1; T++) {
        const PairWin n = pair_tile(a, K, S, FS, FO, T + 1, T + 1 < T1, __shfl_sync(~0u, c.key, 31));
        // bucket of position L: first position s0 (window coordinates, previous
        // tile = 0..31) and end e (coordinates of current + next = 0..63)
        const uint64_t hpc = (uint64_t)c.heads << 32 | hp;
        const uint64_t hcn = (uint64_t)n.heads << 32 | c.heads;
        const uint64_t below = hpc & (lane == 31 ? ~0ull : (2ull << (32 + lane)) - 1);
        const uint64_t above = hcn & ~((2ull << lane) - 1);
        const int s0 = below ? 63 - __clzll((long long)below) : -1;
        const int e = above ? __ffsll((long long)above) - 1 : 64;
        const bool act = s0 >= 0 && e < 64 && e + 32 - s0 <= (int)kSmall && e > (int)lane + 1 && c.lab != kLabDrop;
        // the tile's candidate pairs, dealt out evenly: pair k belongs to the
        // lane L with pre[L] <= k < pre[L] + cand[L], partner position L + d
        const uint32_t cand = act ? (uint32_t)(e - (int)lane - 1) : 0u;
        uint32_t incl = cand;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(~0u, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const uint32_t P = __shfl_sync(~0u, incl, 31);
        if (P) {  // warp-uniform
            W.id[lane] = c.id;
            W.id[32 + lane] = n.id;
            W.lab[lane] = c.lab;
            W.lab[32 + lane] = n.lab;
            W.pre[lane] = incl - cand;
            __syncwarp();
            // This lane's row: its kept partners as a mask over the window.
            // Ids ascend inside a bucket, so the partners past the near-time
            // exclusion start at one position p0 (binary search); dropped
            // entries are cleared by the live mask; only a dense-group member
            // has to clear partners of its own group one by one.
            const uint64_t live = (uint64_t)__ballot_sync(~0u, n.lab != kLabDrop) << 32 |
                                  __ballot_sync(~0u, c.lab != kLabDrop);
            uint64_t keep = 0;
            if (cand && (MODE == 0 || gr.has(c.id >> gshift))) {
                const uint64_t lim = (uint64_t)c.id + a.excl;
                uint32_t lo = lane + 1, hi = (uint32_t)e;
                while (lo < hi) {
                    const uint32_t m = (lo + hi) >> 1;
                    if (W.id[m] <= lim) lo = m + 1;
                    else hi = m;
                }
                keep = live & (((e >= 64 ? 0ull : 1ull << e) - 1) & ~((1ull << lo) - 1));
                if (c.lab != kNone)
                    for (uint64_t m = keep; m; m &= m - 1) {
                        const int y = __ffsll((long long)m) - 1;
                        if (W.lab[y] == c.lab) keep &= ~(1ull << y);
                    }
            }
            const uint32_t cnt = __popcll(keep), g = c.id >> gshift;
            if (MODE != 1) emitted += cnt;
            if (MODE == 0) {
                if (cnt) atomicAdd(gcnt + g, cnt);
            } else if (__any_sync(~0u, cnt != 0)) {
                W.keep[lane] = keep;
                W.base[lane] = !cnt ? 0 : reserve<MODE>(gcur, gpos, g, cnt);
                __syncwarp();
                for (uint32_t k = lane; k < P; k += 32) {
                    uint32_t L = 0;
#pragma unroll
                    for (uint32_t step = 16; step; step >>= 1)
                        if (W.pre[L + step] <= k) L += step;
                    const uint32_t y = L + 1 + (k - W.pre[L]);
                    const uint64_t kl = W.keep[L];
                    if (kl >> y & 1) {
                        const uint32_t i = W.id[L], j = W.id[y];
                        const uint64_t slot = W.base[L] + __popcll(kl & ((1ull << y) - 1));
                        if (MODE == 2) rs.put(i >> gshift, slot, (uint32_t)pack_entry<PT>(i & lmask, j, nbits));
                        else ent[slot] = pack_entry<PT>(i & lmask, j, nbits);
                    }
                }
            }
            __syncwarp();
        }
        hp = c.heads;
        c = n;
    }
    if (MODE != 1 && n_emit) {
        for (int o = 16; o; o >>= 1) emitted += __shfl_down_sync(~0u, emitted, o);
        if (lane == 0 && emitted) atomicAdd(n_emit, emitted);
    }
}

// Medium buckets (more than kSmall entries, fewer than large_min live) are
// split by their number of entries: up to kWarpMed go to one warp each
// (k_medium_warp), larger ones to one CTA each (k_medium_grp).  The CTAs take
// buckets from a shared counter, those of more than kMedFirst entries first,
// so that no large bucket starts last.  Buckets of more than kMedCap live
// members get a launch of their own with the shared memory they need (up to
// kMedHugeCap members).
constexpr uint32_t kWarpMed = 128;
constexpr uint32_t kMedFirst = 1024;
constexpr uint32_t kMedCap = 4096;
constexpr uint32_t kMedHugeCap = 28672;  // 224 KiB of members and labels

struct MedLists {
    const uint4 *warp;  // [*nwarp] buckets of <= kWarpMed entries
    const uint4 *cta;   // [cap]: *nfront from the front, *nback from the back
    const uint4 *huge;  // [*nhuge] buckets of more than kMedCap live members
    const unsigned long long *nwarp, *nfront, *nback, *nhuge;
    uint64_t cap;
    unsigned long long *next, *next_h;  // the CTA launches' work counters, zeroed before each launch
    __device__ __forceinline__ uint4 cta_at(uint64_t v, uint64_t nf) const {
        return v < nf ? cta[v] : cta[cap - 1 - (v - nf)];
    }
};

// Splits the medium list into the warp list and the CTA list (warp-aggregated
// appends; the order inside each class does not matter).
// With count_only, the classes are only counted (the lists are then
// allocated at their sizes).
__global__ void __launch_bounds__(256) k_med_split(const uint4 *__restrict__ medium,
                                                   const unsigned long long *__restrict__ nmedium,
                                                   uint4 *__restrict__ wl, unsigned long long *__restrict__ nw,
                                                   uint4 *__restrict__ cl, uint64_t cap,
                                                   unsigned long long *__restrict__ nf,
                                                   unsigned long long *__restrict__ nb, uint4 *__restrict__ hl,
                                                   unsigned long long *__restrict__ nh, bool count_only) {
    const uint64_t n = *nmedium;
    const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * 32; base < n;
         base += nwarps * 32) {
        const uint64_t x = base + lane;
        uint4 e = make_uint4(0, 0, 0, 0);
        uint32_t cls = 4;
        if (x < n) {
            e = medium[x];
            const uint32_t raw = e.z - e.y;  // e.w: live members
            cls = raw <= kWarpMed ? 0 : e.w > kMedCap ? 3 : raw > kMedFirst ? 1 : 2;
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; k++) {
            const uint32_t m = __ballot_sync(~0u, cls == k);
            if (!m) continue;
            const int leader = __ffs(m) - 1;
            unsigned long long b0 = 0;
            if ((int)lane == leader)
                b0 = atomicAdd(k == 0 ? nw : k == 1 ? nf : k == 2 ? nb : nh, (unsigned long long)__popc(m));
            b0 = __shfl_sync(~0u, b0, leader);
            if (cls == k && !count_only) {
                const uint64_t q = b0 + __popc(m & lt);
                if (k == 0) wl[q] = e;
                else if (k == 1) cl[q] = e;
                else if (k == 2) cl[cap - 1 - q] = e;
                else hl[q] = e;
            }
        }
    }
}

// One CTA per bucket.  Live members (id, group label) are compacted in shared
// memory (mcap of them: dynamic shared memory of 8 mcap bytes); a bucket
// whose members all lie in one dense group has no sparse pairs and is
// skipped.  Rows x are handed to warps one at a time and a warp's lanes take
// the row's partners y > x 32 at a time, so the triangle of pairs is shared
// evenly.  Buckets too large for shared memory fall back to one thread per
// row over global memory.
template <int MODE, typename PT>
__global__ void __launch_bounds__(256) k_medium_grp(EnumArgs a, MedLists ml, bool huge, uint32_t mcap,
                                                    uint32_t gshift, uint32_t nbits, uint32_t *__restrict__ gcnt,
                                                    unsigned long long *__restrict__ gpos, uint32_t *__restrict__ gcur,
                                                    PT *__restrict__ ent, GroupRange gr,
                                                    RegionSink rs = RegionSink{}) {
    extern __shared__ uint32_t med_dyn[];
    uint32_t *s_id = med_dyn, *s_lab = med_dyn + mcap;
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_next, s_mixed;
    __shared__ unsigned long long s_bi;
    const uint64_t nf = huge ? *ml.nhuge : *ml.nfront, n = huge ? nf : nf + *ml.nback;
    unsigned long long *next = huge ? ml.next_h : ml.next;
    const uint32_t lmask = (1u << gshift) - 1, lane = threadIdx.x & 31;
    for (;;) {
        // every thread has read the previous s_bi: the body ends with a barrier
        if (threadIdx.x == 0) s_bi = atomicAdd(next, 1ull);
        __syncthreads();
        const uint64_t bi = s_bi;
        if (bi >= n) break;  // block-uniform
        const uint4 e = huge ? ml.huge[bi] : ml.cta_at(bi, nf);
        const uint32_t *s = a.sid + (uint64_t)e.x * a.N;
        if (e.w > mcap) {  // block-uniform: fallback over global memory
            for (uint32_t x = e.y + threadIdx.x; x < e.z; x += blockDim.x) {
                const uint32_t i = s[x];
                if (a.drop[i] || (MODE == 1 && !gr.has(i >> gshift))) continue;
                uint32_t c = 0;
                for (uint32_t y = x + 1; y < e.z; y++) {
                    const uint32_t j = s[y];
                    c += !a.drop[j] && pair_live(a, i, j);
                }
                if (!c) continue;
                const uint32_t g = i >> gshift;
                if (MODE == 0) {
                    atomicAdd(gcnt + g, c);
                } else {
                    uint64_t o = reserve<MODE>(gcur, gpos, g, c);
                    for (uint32_t y = x + 1; y < e.z; y++) {
                        const uint32_t j = s[y];
                        if (!a.drop[j] && pair_live(a, i, j)) {
                            if (MODE == 2) rs.put(g, o++, (uint32_t)pack_entry<PT>(i & lmask, j, nbits));
                            else ent[o++] = pack_entry<PT>(i & lmask, j, nbits);
                        }
                    }
                }
            }
            __syncthreads();
            continue;
        }
        uint32_t nl = 0;
        if (threadIdx.x == 0) {
            s_next = 0;
            s_mixed = 0;
        }
        for (uint32_t q0 = e.y; q0 < e.z; q0 += blockDim.x) {
            const uint32_t q = q0 + threadIdx.x;
            uint32_t id = 0, live = 0;
            if (q < e.z) {
                id = s[q];
                live = !a.drop[id];
            }
            uint32_t tot;
            const uint32_t pos = block_excl_scan(live, wsum, &tot);
            if (live && nl + pos < mcap) {
                s_id[nl + pos] = id;
                s_lab[nl + pos] = a.label ? __ldg(a.label + id) : kNone;
            }
            nl += tot;
        }
        nl = min(nl, mcap);
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < nl; x += blockDim.x)
            if (s_lab[x] == kNone || s_lab[x] != s_lab[0]) s_mixed = 1;
        __syncthreads();
        if (s_mixed) {  // block-uniform
            // A warp takes R consecutive rows, a lane each (R = nl / 8
            // rounded up, at most 32: every warp of the CTA gets rows of a
            // small bucket too).  Members are in ascending id order, so a
            // row's partners past the near-time exclusion are one contiguous
            // range [y0, nl), found by binary search; only a dense-group
            // member has to skip partners of its own group.  The lanes
            // reserve their rows' slots together, then the warp writes row
            // after row with consecutive stores.
            const uint32_t R = min(32u, max(1u, (nl + 7) / 8));
            for (;;) {
                uint32_t x0 = 0;
                if (lane == 0) x0 = atomicAdd(&s_next, R);
                x0 = __shfl_sync(~0u, x0, 0);
                if (x0 + 1 >= nl) break;  // warp-uniform
                const uint32_t x = x0 + lane;
                uint32_t i = 0, li = kNone, y0 = nl, c = 0;
                if (lane < R && x + 1 < nl) {
                    i = s_id[x];
                    li = s_lab[x];
                    if (MODE != 1 || gr.has(i >> gshift)) {
                        const uint64_t lim = (uint64_t)i + a.excl;
                        uint32_t lo = x + 1, hi = nl;
                        while (lo < hi) {
                            const uint32_t m = (lo + hi) >> 1;
                            if (s_id[m] <= lim) lo = m + 1;
                            else hi = m;
                        }
                        y0 = lo;
                        c = nl - y0;
                        if (li != kNone)
                            for (uint32_t y = y0; y < nl; y++) c -= s_lab[y] == li;
                    }
                }
                const uint32_t g = i >> gshift;
                if (MODE == 0) {
                    if (c) atomicAdd(gcnt + g, c);
                    continue;
                }
                uint64_t base = 0;
                if (c) base = reserve<MODE>(gcur, gpos, g, c);
                for (uint32_t todo = __ballot_sync(~0u, c != 0); todo; todo &= todo - 1) {
                    const int r = __ffs(todo) - 1;
                    const uint32_t ri = __shfl_sync(~0u, i, r), rli = __shfl_sync(~0u, li, r);
                    const uint32_t ry0 = __shfl_sync(~0u, y0, r), rg = ri >> gshift;
                    uint64_t o = __shfl_sync(~0u, base, r);
                    if (rli == kNone) {
                        for (uint32_t y = ry0 + lane; y < nl; y += 32) {
                            const PT e = pack_entry<PT>(ri & lmask, s_id[y], nbits);
                            if (MODE == 2) rs.put(rg, o + (y - ry0), (uint32_t)e);
                            else ent[o + (y - ry0)] = e;
                        }
                    } else {
                        for (uint32_t yb = ry0; yb < nl; yb += 32) {
                            const uint32_t y = yb + lane;
                            const bool keep = y < nl && s_lab[y] != rli;
                            const uint32_t m = __ballot_sync(~0u, keep);
                            if (keep) {
                                const PT e = pack_entry<PT>(ri & lmask, s_id[y], nbits);
                                const uint64_t slot = o + __popc(m & ((1u << lane) - 1));
                                if (MODE == 2) rs.put(rg, slot, (uint32_t)e);
                                else ent[slot] = e;
                            }
                            o += __popc(m);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// One warp per bucket of at most kWarpMed entries: up to four entries a lane,
// live members compacted into the warp's shared-memory slice in id order.
// Each row's partners past the near-time exclusion are one range [y0, nl)
// (binary search); the rows' slots are reserved lane by lane, then the
// warp writes the bucket's pairs of rows outside dense groups as one
// flattened sequence (pair k -> its row by a search over the rows' prefix
// counts), consecutive stores within a row.  Rows of dense-group members
// skip their own group's partners with one ballot per 32 partners.
struct MedWarpSmem {
    uint32_t id[kWarpMed], lab[kWarpMed], pre[kWarpMed], y0[kWarpMed];
    unsigned long long base[kWarpMed];
};

template <int MODE, typename PT>
__global__ void __launch_bounds__(256) k_medium_warp(EnumArgs a, MedLists ml, uint32_t gshift, uint32_t nbits,
                                                     uint32_t *__restrict__ gcnt, unsigned long long *__restrict__ gpos,
                                                     uint32_t *__restrict__ gcur, PT *__restrict__ ent,
                                                     GroupRange gr, RegionSink rs = RegionSink{}) {
    __shared__ MedWarpSmem msm[8];
    MedWarpSmem &W = msm[threadIdx.x / 32];
    const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1, lmask = (1u << gshift) - 1;
    const uint64_t n = *ml.nwarp, nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t bi = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; bi < n; bi += nwarps) {
        const uint4 e = ml.warp[bi];
        const uint32_t *s = a.sid + (uint64_t)e.x * a.N;
        const uint32_t raw = e.z - e.y;
        uint32_t id[4], lab[4];
        bool live[4];
#pragma unroll
        for (int u = 0; u < 4; u++) id[u] = u * 32 + lane < raw ? __ldg(s + e.y + u * 32 + lane) : 0u;
#pragma unroll
        for (int u = 0; u < 4; u++) live[u] = u * 32 + lane < raw && !a.drop[id[u]];
#pragma unroll
        for (int u = 0; u < 4; u++) lab[u] = live[u] && a.label ? __ldg(a.label + id[u]) : kNone;
        __syncwarp();  // the previous bucket's reads of W are done
        uint32_t nl = 0;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t m = __ballot_sync(~0u, live[u]);
            if (live[u]) {
                const uint32_t pos = nl + __popc(m & lt);
                W.id[pos] = id[u];
                W.lab[pos] = lab[u];
            }
            nl += __popc(m);
        }
        __syncwarp();
        if (nl < 2) continue;  // warp-uniform
        const uint32_t l0 = W.lab[0];
        bool mixed = false;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t x = u * 32 + lane;
            if (x < nl) mixed |= W.lab[x] == kNone || W.lab[x] != l0;
        }
        if (!__any_sync(~0u, mixed)) continue;  // one dense group: no sparse pairs
        uint32_t P = 0;  // pairs of rows outside dense groups, in row order
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t x = u * 32 + lane;
            uint32_t c = 0, y0 = nl, i = 0, li = kNone;
            if (x + 1 < nl) {
                i = W.id[x];
                li = W.lab[x];
                if (MODE != 1 || gr.has(i >> gshift)) {
                    const uint64_t lim = (uint64_t)i + a.excl;
                    uint32_t lo = x + 1, hi = nl;
                    while (lo < hi) {
                        const uint32_t m = (lo + hi) >> 1;
                        if (W.id[m] <= lim) lo = m + 1;
                        else hi = m;
                    }
                    y0 = lo;
                    c = nl - y0;
                    if (li != kNone)
                        for (uint32_t y = y0; y < nl; y++) c -= W.lab[y] == li;
                }
            }
            const uint32_t g = i >> gshift;
            if (MODE == 0) {
                if (c) atomicAdd(gcnt + g, c);
                continue;
            }
            unsigned long long b = 0;
            if (c) b = reserve<MODE>(gcur, gpos, g, c);
            const uint32_t cu = li == kNone ? c : 0u;
            uint32_t inc = cu;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(~0u, inc, o);
                if ((int)lane >= o) inc += y;
            }
            W.pre[x] = P + inc - cu;
            W.y0[x] = y0;
            W.base[x] = b;
            P += __shfl_sync(~0u, inc, 31);
            // rows of dense-group members: partners of other groups only
            for (uint32_t todo = __ballot_sync(~0u, li != kNone && c != 0); todo; todo &= todo - 1) {
                const int r = __ffs(todo) - 1;
                const uint32_t ri = __shfl_sync(~0u, i, r), rli = __shfl_sync(~0u, li, r);
                const uint32_t ry0 = __shfl_sync(~0u, y0, r);
                unsigned long long o = __shfl_sync(~0u, b, r);
                for (uint32_t yb = ry0; yb < nl; yb += 32) {
                    const uint32_t y = yb + lane;
                    const bool keep = y < nl && W.lab[y] != rli;
                    const uint32_t m = __ballot_sync(~0u, keep);
                    if (keep) {
                        const PT ev = pack_entry<PT>(ri & lmask, W.id[y], nbits);
                        const unsigned long long slot = o + __popc(m & lt);
                        if (MODE == 2) rs.put(ri >> gshift, slot, (uint32_t)ev);
                        else ent[slot] = ev;
                    }
                    o += __popc(m);
                }
            }
        }
        if (MODE == 0) continue;
        __syncwarp();
        // pair k: the last row x < nl - 1 with pre[x] <= k (rows without
        // pairs share their successor's prefix, so x has pairs left)
        for (uint32_t k = lane; k < P; k += 32) {
            uint32_t x = 0;
#pragma unroll
            for (uint32_t step = kWarpMed / 2; step; step >>= 1)
                if (x + step + 1 < nl && W.pre[x + step] <= k) x += step;
            const uint32_t d = k - W.pre[x], i = W.id[x];
            const PT ev = pack_entry<PT>(i & lmask, W.id[W.y0[x] + d], nbits);
            if (MODE == 2) rs.put(i >> gshift, W.base[x] + d, (uint32_t)ev);
            else ent[W.base[x] + d] = ev;
        }
    }
}

struct VoteArgs {
    const uint64_t *goff;
    uint64_t ngroups, N;
    uint64_t g_lo, g_hi, ebase;  // the groups of this pass and the buffer offset of group g_lo
    uint32_t gshift, nbits, v, vcap;
    uint32_t *sp_cnt;
    uint64_t *sp_start;
    uint32_t *sp_j;
    uint8_t *sp_v;
    uint64_t sp_cap;
    unsigned long long *sp_cursor;
    uint2 *long_rows;  // (row, candidate bound) for rows voted one CTA each
    unsigned long long *n_long;
    uint64_t long_cap;
    // single-pass layout (rcnt != nullptr): group g's first rcap entries at
    // g * rcap, the rest in the overflow list (sorted by group) from ostart[g]
    const uint32_t *rcnt;
    uint32_t rcap;
    const unsigned long long *ovf;
    const uint64_t *ostart;
};

// Where group g's entries are: base e0 and count n.
__device__ __forceinline__ void group_span(const VoteArgs &A, uint64_t g, uint64_t &e0, uint64_t &n) {
    if (A.rcnt) {
        e0 = g * A.rcap;
        n = A.rcnt[g];
    } else {
        e0 = A.goff[g] - A.ebase;
        n = A.goff[g + 1] - A.goff[g];
    }
}

// Entries of group g below `lim` lie at e0 + x; entries from lim to n are in
// the overflow list (single pass only).  Loads are predicated, not branched,
// so a batch of them stays in flight together.
__device__ __forceinline__ uint64_t region_lim(const VoteArgs &A, uint64_t n) {
    return A.rcnt ? min(n, (uint64_t)A.rcap) : n;
}

template <typename PT>
__device__ __forceinline__ PT entry_at(const VoteArgs &A, const PT *__restrict__ ent, uint64_t g, uint64_t e0,
                                       uint64_t lim, uint64_t x, bool stream = false) {
    if (x < lim) return stream ? __ldcs(ent + e0 + x) : ent[e0 + x];
    return (PT)(uint32_t)A.ovf[A.ostart[g] + (x - lim)];
}

// Hash insert for the row votes (key j+1, 0 = empty), 32-bit counts.
__device__ __forceinline__ bool vadd(uint32_t *K, uint32_t *C, uint32_t slots, uint32_t j) {
    const uint32_t want = j + 1;
    uint32_t h = row_hash(j) & (slots - 1);
    for (uint32_t probe = 0; probe < slots; probe++) {
        uint32_t kk = K[h];
        if (kk == 0) {
            kk = atomicCAS(K + h, 0u, want);
            if (kk == 0) kk = want;
        }
        if (kk == want) {
            atomicAdd(C + h, 1u);
            return true;
        }
        h = (h + 1) & (slots - 1);
    }
    return false;
}

// A row group's pairs are counted in one shared-memory hash of >= 2n slots
// when n <= vcap (larger groups: one CTA per row).  The expected pairs per
// group (`group_pairs`, default 1024) sets the group size 2^gshift rows, and
// vcap is twice the power of two above it: larger groups mean fewer
// concurrent write frontiers in the emission pass, smaller ones more resident
// CTAs in the vote.
constexpr uint32_t kVTargetDefault = 1024;
// Counting filter in front of the hash: 16-bit counters (never wrap: a group
// holds at most vcap <= 16384 entries) indexed by a second hash of the entry.
// An entry whose counter is below v cannot have v copies, so only the few
// that pass are counted exactly.
constexpr uint32_t kVFilter = 8192;
constexpr int kVRegs = 8;  // entries per thread held in registers (groups of up to 2048 at 256 threads)

template <typename PT>
size_t group_vote_smem(uint32_t vcap) {
    return (size_t)2 * vcap * sizeof(PT) + (size_t)2 * vcap / 4 * 4 + (size_t)kVFilter * 2;
}

// Slot of a key in a table of 2^lg slots: multiplicative (Fibonacci) hashing,
// top lg bits of key * 2^w / golden ratio; 64-bit keys are mixed first.
__device__ __forceinline__ uint32_t ghash(uint32_t key, uint32_t lg) { return (key * 0x9E3779B1u) >> (32 - lg); }
__device__ __forceinline__ uint32_t ghash(unsigned long long key, uint32_t lg) {
    return (uint32_t)(mix64(key) >> (64 - lg));
}
// The counting filter's index: another multiplier, so that filter and hash
// collisions are independent.
__device__ __forceinline__ uint32_t fhash(uint32_t key, uint32_t lg) { return (key * 0x85EBCA6Bu) >> (32 - lg); }
__device__ __forceinline__ uint32_t fhash(unsigned long long key, uint32_t lg) {
    return (uint32_t)((key * 0xC2B2AE3D27D4EB4Full) >> (64 - lg));
}

// One CTA per group: every entry (local row, j) of the group counted in one
// shared-memory hash of >= 2n slots; entries seen at least v times are the
// group's detections, ordered by (local row, j) -- i.e. by (i, j) -- by rank.
// One row group of the vote (see k_group_vote): counting filter, exact counts
// of the entries that pass, kept pairs in (i, j) order.
#define VOTE_FOR_ENTRIES(raw, BODY)                                                   \
    if (regs) {                                                                       \
        _Pragma("unroll") for (int u_ = 0; u_ < kVRegs; u_++) {                      \
            if (threadIdx.x + (uint64_t)u_ * blockDim.x >= n) continue;              \
            const PT raw = cur[u_];                                                   \
            if ((uint32_t)(raw >> A.nbits) - r0 >= r1 - r0) continue;                 \
            BODY                                                                      \
        }                                                                             \
    } else {                                                                          \
        for (uint64_t x_ = threadIdx.x; x_ < n; x_ += blockDim.x) {                   \
            const PT raw = entry_at(A, ent, g, e0, region_lim(A, n), x_);             \
            if ((uint32_t)(raw >> A.nbits) - r0 >= r1 - r0) continue;                 \
            BODY                                                                      \
        }                                                                             \
    }

template <typename PT>
__device__ __forceinline__ void vote_one(const VoteArgs &A, const PT *__restrict__ ent, uint64_t g, uint64_t e0,
                                         uint64_t n, uint32_t r0, uint32_t r1, const PT (&cur)[kVRegs], PT *K,
                                         uint32_t *C, uint32_t *F,
                                         uint32_t &s_pass, uint32_t *wsum, unsigned long long &s_b0, PT jmask) {
    const bool regs = n <= (uint64_t)kVRegs * blockDim.x;
        if (n < A.v) return;  // block-uniform
        const uint64_t row0 = g << A.gshift;
        if (n > A.vcap) {  // every row of the group is voted one CTA each
            for (uint32_t r = threadIdx.x; r < (1u << A.gshift); r += blockDim.x) {
                if (row0 + r >= A.N) break;
                unsigned long long q = atomicAdd(A.n_long, 1ull);
                if (q < A.long_cap) A.long_rows[q] = make_uint2((uint32_t)(row0 + r), (uint32_t)n);
            }
            return;
        }
        // 1. counting filter
        uint32_t fc = 64, flg = 6;
        while (fc < 2 * n && fc < kVFilter) fc <<= 1, flg++;
        for (uint32_t x = threadIdx.x; x < fc / 2; x += blockDim.x) F[x] = 0;
        if (threadIdx.x == 0) s_pass = 0;
        __syncthreads();
        VOTE_FOR_ENTRIES(raw, {
            const uint32_t f = fhash(raw, flg);
            atomicAdd(F + (f >> 1), 1u << (16 * (f & 1)));
        })
        __syncthreads();
        uint32_t mine = 0;
        VOTE_FOR_ENTRIES(raw, {
            const uint32_t f = fhash(raw, flg);
            mine += (F[f >> 1] >> (16 * (f & 1)) & 0xFFFF) >= A.v;
        })
        if (mine) atomicAdd(&s_pass, mine);
        __syncthreads();
        const uint32_t npass = s_pass;
        if (npass < A.v) {  // block-uniform: nothing can reach v votes
            __syncthreads();
            return;
        }
        // 2. exact counts of the entries that pass, in a hash of >= 2 npass slots
        uint32_t slots = 64, lg = 6;
        while (slots < 2 * npass) slots <<= 1, lg++;
        for (uint32_t x = threadIdx.x; x < slots; x += blockDim.x) K[x] = 0;
        for (uint32_t x = threadIdx.x; x < slots / 4; x += blockDim.x) C[x] = 0;
        __syncthreads();
        VOTE_FOR_ENTRIES(raw, {
            const uint32_t f = fhash(raw, flg);
            if ((F[f >> 1] >> (16 * (f & 1)) & 0xFFFF) < A.v) continue;
            const PT want = raw + 1;
            uint32_t h = ghash(want, lg);
            for (uint32_t probe = 0; probe < slots; probe++) {
                PT kk = K[h];
                if (kk == 0) {
                    kk = atomicCAS(K + h, (PT)0, want);
                    if (kk == 0) kk = want;
                }
                if (kk == want) {
                    atomicAdd(C + (h >> 2), 1u << (8 * (h & 3)));
                    break;
                }
                h = (h + 1) & (slots - 1);
            }
        })
        __syncthreads();
        // kept entries compacted to the front of each warp's slot segment (a
        // kept slot's new position never exceeds its old one, and every lane
        // reads its slot before the ballot, so no unread slot is overwritten)
        const uint32_t nw = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x & 31;
        const uint32_t seg = slots / nw, lo = warp * seg;
        uint32_t wn = 0;
        for (uint32_t base = lo; base < lo + seg; base += 32) {
            const uint32_t x = base + lane;
            PT kk = 0;
            uint32_t cc = 0;
            if (x < lo + seg) {
                kk = K[x];
                cc = (C[x >> 2] >> (8 * (x & 3))) & 0xFF;
            }
            const bool keep = kk != 0 && cc >= A.v;
            const uint32_t m = __ballot_sync(~0u, keep);
            if (keep) {
                const uint32_t pos = lo + wn + __popc(m & ((1u << lane) - 1));
                K[pos] = kk - 1;
                reinterpret_cast<uint8_t *>(C)[pos] = (uint8_t)cc;
            }
            wn += __popc(m);
        }
        if (lane == 0) wsum[warp] = wn;
        __syncthreads();
        uint32_t nk = 0;
        for (uint32_t w = 0; w < nw; w++) nk += wsum[w];
        if (!nk) {  // block-uniform
            __syncthreads();
            return;
        }
        if (threadIdx.x == 0) s_b0 = atomicAdd(A.sp_cursor, (unsigned long long)nk);
        __syncthreads();
        const uint64_t b0 = s_b0;
        const uint8_t *V = reinterpret_cast<const uint8_t *>(C);
        // each kept entry's rank among the group's kept entries = its place in (i, j) order
        for (uint32_t w = 0; w < nw; w++) {
            for (uint32_t q = threadIdx.x; q < wsum[w]; q += blockDim.x) {
                const uint32_t x = w * seg + q;
                const PT kx = K[x];
                uint32_t rank = 0, first = 1;
                for (uint32_t w2 = 0; w2 < nw; w2++) {
                    const PT *Kw = K + w2 * seg;
                    for (uint32_t y = 0, ny = wsum[w2]; y < ny; y++) {
                        const PT ky = Kw[y];
                        rank += ky < kx;
                        first &= (uint32_t)((ky >> A.nbits) != (kx >> A.nbits) || ky >= kx);
                    }
                }
                const uint64_t i = row0 + (uint32_t)(kx >> A.nbits);
                if (b0 + nk <= A.sp_cap) {
                    A.sp_j[b0 + rank] = (uint32_t)(kx & jmask);
                    A.sp_v[b0 + rank] = V[x];
                }
                atomicAdd(A.sp_cnt + i, 1u);
                if (first) A.sp_start[i] = b0 + rank;  // the row's smallest j
            }
        }
        __syncthreads();
}
#undef VOTE_FOR_ENTRIES

template <typename PT>
__global__ void __launch_bounds__(256) k_group_vote(VoteArgs A, const PT *__restrict__ ent,
                                                    const uint2 *__restrict__ list,
                                                    const unsigned long long *__restrict__ nlist) {
    extern __shared__ unsigned long long vsm_raw[];
    PT *K = reinterpret_cast<PT *>(vsm_raw);                             // [<= 2 vcap] keys (entry + 1)
    uint32_t *C = reinterpret_cast<uint32_t *>(K + 2 * A.vcap);          // [<= 2 vcap / 4] byte counts
    uint32_t *F = C + 2 * A.vcap / 4;                                    // [kVFilter / 2] 16-bit counters
    __shared__ uint32_t s_pass;
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long s_b0;
    const PT jmask = ((PT)1 << A.nbits) - 1;
    // A group's entries stay in registers (kVRegs per thread) when they fit,
    // and the next group's are loaded while this one is counted.
    PT cur[kVRegs], nxt[kVRegs];
    uint64_t e0 = 0, n = 0, e0n = 0, nn = 0;
    auto fetch = [&](uint64_t gg, PT (&buf)[kVRegs], uint64_t &s0, uint64_t &cnt) {
        s0 = 0;
        cnt = 0;
        if (gg < A.ngroups) group_span(A, gg, s0, cnt);
        const bool regs = cnt >= A.v && cnt <= A.vcap && cnt <= (uint64_t)kVRegs * blockDim.x;
#pragma unroll
        for (int u = 0; u < kVRegs; u++) {
            const uint64_t x = threadIdx.x + (uint64_t)u * blockDim.x;
            buf[u] = regs && x < cnt ? entry_at(A, ent, gg, s0, region_lim(A, cnt), x, true) : (PT)0;
        }
    };
    const uint64_t count = list ? *nlist : A.ngroups;
    auto gid = [&](uint64_t k) { return list ? (uint64_t)list[k].x : k; };
    // rows [r0, r1) of the group (all of them without a list)
    auto rng = [&](uint64_t k) { return list ? list[k].y : (1u << A.gshift); };
    fetch(blockIdx.x < count ? gid(blockIdx.x) : A.ngroups, cur, e0, n);
    for (uint64_t k = blockIdx.x; k < count; k += gridDim.x) {
        fetch(k + gridDim.x < count ? gid(k + gridDim.x) : A.ngroups, nxt, e0n, nn);
        const uint32_t rr = rng(k);
        vote_one(A, ent, gid(k), e0, n, rr >> 16, rr & 0xFFFF, cur, K, C, F, s_pass, wsum, s_b0, jmask);
#pragma unroll
        for (int u = 0; u < kVRegs; u++) cur[u] = nxt[u];
        e0 = e0n;
        n = nn;
    }
}

// Warp-per-group vote for the common case, no block barriers: each warp has
// its own counting filter (kWF 16-bit counters) and a small exact hash (kWS
// slots) in shared memory.  Groups too large for them (more than kWF / 2
// entries, or more than kWS / 2 entries passing the filter) are appended to
// `slow` for the block kernel; groups beyond vcap are split into long rows as
// the block kernel does.
constexpr uint32_t kWF = 4096, kWS = 256, kVW = 6;  // kVW warps per CTA: four CTAs per SM fit

template <typename PT>
constexpr size_t warp_vote_smem() {
    return (size_t)kVW * (kWF * 2 + kWS * sizeof(PT) + kWS);
}

template <typename PT>
__global__ void __launch_bounds__(kVW * 32) k_warp_vote(VoteArgs A, const PT *__restrict__ ent, uint2 *__restrict__ slow,
                                                   unsigned long long *__restrict__ nslow) {
    extern __shared__ unsigned long long wv_raw[];
    const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    char *base = reinterpret_cast<char *>(wv_raw) + (size_t)warp * (kWF * 2 + kWS * sizeof(PT) + kWS);
    PT *K = reinterpret_cast<PT *>(base);                                // [kWS] keys (entry + 1)
    uint32_t *F = reinterpret_cast<uint32_t *>(base + kWS * sizeof(PT)); // [kWF / 2] 16-bit counters
    uint8_t *V = reinterpret_cast<uint8_t *>(F + kWF / 2);               // [kWS] counts
    const PT jmask = ((PT)1 << A.nbits) - 1;
    const uint32_t lt = (1u << lane) - 1;
    for (uint64_t g = A.g_lo + (uint64_t)blockIdx.x * kVW + warp; g < A.g_hi; g += (uint64_t)gridDim.x * kVW) {
        uint64_t e0, n;
        group_span(A, g, e0, n);
        if (n < A.v) continue;  // warp-uniform
        const uint64_t lim = region_lim(A, n);
        const uint64_t row0 = g << A.gshift;
        if (n > A.vcap) {  // every row of the group is voted one CTA each
            for (uint32_t r = lane; r < (1u << A.gshift); r += 32) {
                if (row0 + r >= A.N) break;
                const unsigned long long q = atomicAdd(A.n_long, 1ull);
                if (q < A.long_cap) A.long_rows[q] = make_uint2((uint32_t)(row0 + r), (uint32_t)n);
            }
            continue;
        }
        // a group larger than the filter is voted in parts: row ranges of about
        // kWF / 4 entries each (one part when it fits)
        const uint32_t rows = 1u << A.gshift;
        const uint32_t P = n <= kWF / 2 ? 1u : min(min(rows, 8u), (uint32_t)((n + kWF / 4 - 1) / (kWF / 4)));
        uint32_t pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (P > 1) {
            for (uint32_t x0 = lane; x0 < n; x0 += 8 * 32) {
                PT b8[8];
#pragma unroll
                for (int u = 0; u < 8; u++) b8[u] = x0 + 32 * u < lim ? ent[e0 + x0 + 32 * u] : x0 + 32 * u < n ? entry_at(A, ent, g, e0, lim, x0 + 32 * u) : (PT)0;
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const uint32_t part = x0 + 32 * u < n ? (uint32_t)(b8[u] >> A.nbits) * P / rows : 8u;
#pragma unroll
                    for (int q = 0; q < 8; q++) pc[q] += part == (uint32_t)q;
                }
            }
#pragma unroll
            for (int q = 0; q < 8; q++)
#pragma unroll
                for (int o = 16; o; o >>= 1) pc[q] += __shfl_xor_sync(~0u, pc[q], o);
        } else {
            pc[0] = (uint32_t)n;
        }
        bool fits = true;
#pragma unroll
        for (int q = 0; q < 8; q++) fits &= pc[q] <= kWF / 2;
        if (!fits) {  // uneven rows: the whole group to the block kernel
            if (lane == 0) slow[atomicAdd(nslow, 1ull)] = make_uint2((uint32_t)g, rows);
            continue;
        }
        for (uint32_t p = 0; p < P; p++) {
        // part of row r is r * P / rows, so part p holds rows [ceil(p rows / P), ceil((p + 1) rows / P))
        const uint32_t r0 = (p * rows + P - 1) / P, r1 = ((p + 1) * rows + P - 1) / P, np = pc[min(p, 7u)];
        if (np < A.v) continue;
        // 1. counting filter
        uint32_t fc = 64, flg = 6;
        while (fc < 2 * np) fc <<= 1, flg++;
        for (uint32_t x = lane; x < fc / 2; x += 32) F[x] = 0;
        __syncwarp();
        // entries in batches of 8 per lane, all loads of a batch issued before its atomics
        for (uint32_t x0 = lane; x0 < n; x0 += 8 * 32) {
            PT b8[8];
#pragma unroll
            for (int u = 0; u < 8; u++) b8[u] = x0 + 32 * u < lim ? ent[e0 + x0 + 32 * u] : x0 + 32 * u < n ? entry_at(A, ent, g, e0, lim, x0 + 32 * u) : (PT)0;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (x0 + 32 * u < n && (uint32_t)(b8[u] >> A.nbits) - r0 < r1 - r0) {
                    const uint32_t f = fhash(b8[u], flg);
                    atomicAdd(F + (f >> 1), 1u << (16 * (f & 1)));
                }
        }
        __syncwarp();
        uint32_t npass = 0;
        for (uint32_t x0 = lane; x0 < n; x0 += 8 * 32) {
            PT b8[8];
#pragma unroll
            for (int u = 0; u < 8; u++) b8[u] = x0 + 32 * u < lim ? ent[e0 + x0 + 32 * u] : x0 + 32 * u < n ? entry_at(A, ent, g, e0, lim, x0 + 32 * u) : (PT)0;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (x0 + 32 * u < n && (uint32_t)(b8[u] >> A.nbits) - r0 < r1 - r0) {
                    const uint32_t f = fhash(b8[u], flg);
                    npass += (F[f >> 1] >> (16 * (f & 1)) & 0xFFFF) >= A.v;
                }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) npass += __shfl_xor_sync(~0u, npass, o);
        if (npass < A.v) continue;  // nothing can reach v votes
        if (npass > kWS / 2) {  // this part's rows to the block kernel
            if (lane == 0) slow[atomicAdd(nslow, 1ull)] = make_uint2((uint32_t)g, r0 << 16 | r1);
            continue;
        }
        // 2. exact counts of the passing entries
        uint32_t slots = 32, lg = 5;
        while (slots < 2 * npass) slots <<= 1, lg++;
        for (uint32_t x = lane; x < slots; x += 32) {
            K[x] = 0;
            V[x] = 0;
        }
        __syncwarp();
        for (uint32_t x0 = lane; x0 < n; x0 += 8 * 32) {
            PT b8[8];
#pragma unroll
            for (int u = 0; u < 8; u++)
                b8[u] = x0 + 32 * u < lim ? (p + 1 == P ? __ldcs(ent + e0 + x0 + 32 * u) : ent[e0 + x0 + 32 * u])
                        : x0 + 32 * u < n ? entry_at(A, ent, g, e0, lim, x0 + 32 * u) : (PT)0;
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (x0 + 32 * u >= n || (uint32_t)(b8[u] >> A.nbits) - r0 >= r1 - r0) continue;
                const uint32_t f = fhash(b8[u], flg);
                if ((F[f >> 1] >> (16 * (f & 1)) & 0xFFFF) < A.v) continue;
                const PT want = b8[u] + 1;
                uint32_t h = ghash(want, lg);
                for (uint32_t probe = 0; probe < slots; probe++) {
                    PT kk = K[h];
                    if (kk == 0) {
                        kk = atomicCAS(K + h, (PT)0, want);
                        if (kk == 0) kk = want;
                    }
                    if (kk == want) {
                        atomicAdd(reinterpret_cast<uint32_t *>(V) + (h >> 2), 1u << (8 * (h & 3)));
                        break;
                    }
                    h = (h + 1) & (slots - 1);
                }
            }
        }
        __syncwarp();
        // 3. kept entries compacted to the front (positions never pass the read point)
        uint32_t nk = 0;
        for (uint32_t b = 0; b < slots; b += 32) {
            const uint32_t x = b + lane;
            const PT kk = K[x];
            const uint32_t cc = V[x];
            const bool keep = kk != 0 && cc >= A.v;
            const uint32_t m = __ballot_sync(~0u, keep);
            if (keep) {
                const uint32_t pos = nk + __popc(m & lt);
                K[pos] = kk - 1;
                V[pos] = (uint8_t)cc;
            }
            nk += __popc(m);
        }
        __syncwarp();
        if (!nk) continue;
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(A.sp_cursor, (unsigned long long)nk);
        b0 = __shfl_sync(~0u, b0, 0);
        for (uint32_t q = lane; q < nk; q += 32) {
            const PT kx = K[q];
            uint32_t rank = 0, first = 1;
            for (uint32_t y = 0; y < nk; y++) {
                const PT ky = K[y];
                rank += ky < kx;
                first &= (uint32_t)((ky >> A.nbits) != (kx >> A.nbits) || ky >= kx);
            }
            const uint64_t i = row0 + (uint32_t)(kx >> A.nbits);
            if (b0 + nk <= A.sp_cap) {
                A.sp_j[b0 + rank] = (uint32_t)(kx & jmask);
                A.sp_v[b0 + rank] = V[q];
            }
            atomicAdd(A.sp_cnt + i, 1u);
            if (first) A.sp_start[i] = b0 + rank;
        }
        __syncwarp();
        }  // parts
    }
}

// Long rows: one CTA per row, the row's entries filtered out of its group's
// region; hash of pow2 >= 2n slots in shared memory (up to kRowBlockSlots)
// or in global scratch at gscratch + gofs[r].
template <typename PT>
__global__ void __launch_bounds__(512) k_long_vote(VoteArgs A, const PT *__restrict__ ent,
                                                   const uint2 *__restrict__ rows, uint64_t nrows,
                                                   uint32_t *__restrict__ gscratch, const uint64_t *__restrict__ gofs) {
    extern __shared__ uint32_t sm_row[];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_nk;
    __shared__ unsigned long long s_b0;
    const PT jmask = ((PT)1 << A.nbits) - 1;
    for (uint64_t rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
        const uint32_t i = rows[rr].x;
        const uint64_t bound = rows[rr].y;
        uint32_t slots = 32;
        while (slots < 2 * bound) slots <<= 1;
        uint32_t *K = sm_row, *C;
        if (slots <= kRowBlockSlots) {
            C = sm_row + slots;
        } else {
            K = gscratch + gofs[rr];
            C = K + slots;
        }
        for (uint32_t x = threadIdx.x; x < slots; x += blockDim.x) K[x] = 0, C[x] = 0;
        __syncthreads();
        const uint64_t g = i >> A.gshift;
        const uint32_t local = i & ((1u << A.gshift) - 1);
        uint64_t e0, n;
        group_span(A, g, e0, n);
        for (uint64_t x = threadIdx.x; x < n; x += blockDim.x) {
            const PT en = entry_at(A, ent, g, e0, region_lim(A, n), x);
            if ((uint32_t)(en >> A.nbits) == local) vadd(K, C, slots, (uint32_t)(en & jmask));
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nk = 0;
        __syncthreads();
        for (uint32_t base = 0; base < slots; base += blockDim.x) {
            const uint32_t x = base + threadIdx.x;
            uint32_t cc = 0, kk = 0;
            if (x < slots) {
                cc = C[x];
                kk = K[x];
            }
            const uint32_t keep = kk != 0 && cc >= A.v;
            uint32_t tot;
            const uint32_t pos = s_nk + block_excl_scan(keep, wsum, &tot);
            if (keep) {
                K[pos] = kk - 1;
                C[pos] = cc;
            }
            __syncthreads();
            if (threadIdx.x == 0) s_nk += tot;
            __syncthreads();
        }
        const uint32_t nk = s_nk;
        if (nk) {
            if (threadIdx.x == 0) {
                s_b0 = atomicAdd(A.sp_cursor, (unsigned long long)nk);
                A.sp_cnt[i] = nk;
                A.sp_start[i] = s_b0;
            }
            __syncthreads();
            if (s_b0 + nk <= A.sp_cap) row_write_sorted(K, C, nk, threadIdx.x, blockDim.x, A.sp_j, A.sp_v, s_b0);
        }
        __syncthreads();
    }
}

// Dense groups, count pass for the row layout: detections per row, one
// atomic per (row, tile).
// Tiles of groups whose cluster masks overflowed (gover[tile_grp[ti]] != 0)
// only; the others are voted by k_dense_rowcount_mask.
__global__ void __launch_bounds__(256) k_dense_rowcount(const DenseTile *__restrict__ tiles, uint64_t ntiles,
                                                        const uint32_t *__restrict__ GT, const uint32_t *__restrict__ ids,
                                                        uint64_t nm, uint32_t nb, uint32_t v, uint32_t excl,
                                                        uint32_t *__restrict__ dense_cnt, uchar4 *__restrict__ tv,
                                                        const uint32_t *__restrict__ tile_grp,
                                                        const uint32_t *__restrict__ gover) {
    extern __shared__ uint32_t sd[];
    uint32_t *sA = sd, *sB = sd + (size_t)nb * kDT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        if (!gover[tile_grp[ti]]) continue;  // block-uniform
        const DenseTile T = tiles[ti];
        const uint32_t a0 = T.g0 + T.ta * kDT, b0 = T.g0 + T.tb * kDT;
        const uint32_t na = min((uint32_t)kDT, T.n - T.ta * kDT), nbb = min((uint32_t)kDT, T.n - T.tb * kDT);
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < nb * kDT; x += blockDim.x) {
            const uint32_t t = x / kDT, c = x % kDT;
            sA[x] = c < na ? GT[(uint64_t)t * nm + a0 + c] : 0xFFFFFFFFu;
            sB[x] = c < nbb ? GT[(uint64_t)t * nm + b0 + c] : 0xFFFFFFFEu;
        }
        __syncthreads();
        uint32_t acc[4][4] = {};
        for (uint32_t t = 0; t < nb; t++) {
            const uint4 av = *reinterpret_cast<const uint4 *>(sA + t * kDT + ty * 4);
            const uint4 bv = *reinterpret_cast<const uint4 *>(sB + t * kDT + tx * 4);
            const uint32_t A4[4] = {av.x, av.y, av.z, av.w}, B4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int w = 0; w < 4; w++) acc[u][w] += A4[u] == B4[w];
        }
        // the tile's votes, kept for the emit pass: row ty*4+u, columns tx*4 .. +3
#pragma unroll
        for (int u = 0; u < 4; u++)
            tv[ti * (kDT * kDT / 4) + (ty * 4 + u) * (kDT / 4) + tx] =
                make_uchar4((uint8_t)acc[u][0], (uint8_t)acc[u][1], (uint8_t)acc[u][2], (uint8_t)acc[u][3]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t ga = T.ta * kDT + ty * 4 + u;
            uint32_t c = 0;
            const uint32_t i = ga < T.n ? ids[T.g0 + ga] : 0;
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const uint32_t gb = T.tb * kDT + tx * 4 + w;
                if (ga < T.n && gb < T.n && ga < gb && acc[u][w] >= v && ids[T.g0 + gb] - i > excl) ++c;
            }
#pragma unroll
            for (int d = 8; d; d >>= 1) c += __shfl_down_sync(~0u, c, d, 16);
            if (tx == 0 && c) atomicAdd(dense_cnt + i, c);
        }
    }
}

// ---- dense votes from cluster masks
//
// Inside one dense group, the members sharing a key in table t form a
// cluster; votes(i, j) is the number of tables in which i and j fall in the
// same cluster.  Clusters of at least the group's threshold get one bit
// column each (at most kClW * 32 per group): the tables where i and j share
// such a cluster number popc(mask_i & mask_j).  The pairs of the smaller
// clusters are added one by one into the tile votes.  Both parts are exact,
// so their sum is the vote.  The threshold is a power of two from kClT up,
// chosen per group from a histogram of its cluster sizes: the one with the
// fewest mask words per member pair plus enumerated pairs (weighted
// kClEnum), among those that leave at most kClW * 32 columns.
constexpr uint32_t kClT = 64;
constexpr uint32_t kClW = 32;
constexpr uint32_t kClBins = 18;  // cluster sizes 64 * 2^k .. 64 * 2^(k+1) - 1
constexpr double kClEnum = 64.0;  // an enumerated pair (global atomic) against one mask word of a member pair

struct DenseGroup {
    uint32_t g0, n, t0, nt;  // first member, members, first tile, tiles per side
};

// comp[t * nm + k] = t : 8 | key : 32 | k : 24 (member k of table t)
__global__ void k_clu_comp(const uint32_t *__restrict__ GT, uint64_t nm, uint32_t nb,
                           unsigned long long *__restrict__ comp) {
    const uint64_t n = (uint64_t)nb * nm;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x)
        comp[e] = (unsigned long long)(e / nm) << 56 | (unsigned long long)GT[e] << 24 | (e % nm);
}

// flag[e] = 1 where a cluster starts in the sorted list: a new (table, key),
// or a new group within the same (table, key).
__global__ void k_clu_mark(const unsigned long long *__restrict__ comp, uint64_t n, const uint32_t *__restrict__ mg,
                           uint32_t *__restrict__ flag) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = comp[e];
        uint32_t f = 1;
        if (e) {
            const unsigned long long y = comp[e - 1];
            f = (x >> 24) != (y >> 24) || mg[x & 0xFFFFFF] != mg[y & 0xFFFFFF];
        }
        flag[e] = f;
    }
}

__global__ void k_clu_starts(const uint32_t *__restrict__ flag, const uint64_t *__restrict__ cid, uint64_t n,
                             const uint64_t *__restrict__ ncl, uint64_t *__restrict__ cst) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        if (flag[e]) cst[cid[e]] = e;
        if (e == 0) cst[*ncl] = n;
    }
}

// Per group: clusters and their pairs by size class (sizes of at least kClT).
__global__ void k_clu_hist(const unsigned long long *__restrict__ comp, const uint64_t *__restrict__ cst,
                           const uint64_t *__restrict__ ncl, const uint32_t *__restrict__ mg,
                           uint32_t *__restrict__ hcnt, unsigned long long *__restrict__ hpairs) {
    const uint64_t nc = *ncl;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t sz = cst[c + 1] - cst[c];
        if (sz < kClT) continue;
        const uint32_t g = mg[comp[cst[c]] & 0xFFFFFF];
        const uint32_t bin = min(kClBins - 1, (uint32_t)(63 - __clzll((long long)(sz / kClT))));
        atomicAdd(hcnt + (uint64_t)g * kClBins + bin, 1u);
        atomicAdd(hpairs + (uint64_t)g * kClBins + bin, (unsigned long long)(sz * (sz - 1) / 2));
    }
}

// Per group: the mask threshold kClT * 2^k of least estimated cost (see
// above); gover marks a group that direct key comparison votes for less (b
// comparisons per member pair, about two thirds of a mask word each).
__global__ void k_clu_thr(const DenseGroup *__restrict__ G, uint64_t ngroups, uint32_t nb,
                          const uint32_t *__restrict__ hcnt, const unsigned long long *__restrict__ hpairs,
                          uint32_t *__restrict__ gthr, uint32_t *__restrict__ gover) {
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const double mp = (double)G[g].n * (G[g].n - 1) / 2;
        const uint32_t *h = hcnt + g * kClBins;
        const unsigned long long *hp = hpairs + g * kClBins;
        double best = 0, below = 0;  // enumerated pairs of the classes under threshold k
        uint32_t bk = kClBins + 1;
        for (uint32_t k = 0; k <= kClBins; k++) {
            uint64_t cols = 0;
            for (uint32_t q = k; q < kClBins; q++) cols += h[q];
            if (cols <= kClW * 32) {
                const double cost = mp * (double)((cols + 31) / 32) + kClEnum * below;
                if (bk > kClBins || cost < best) {
                    best = cost;
                    bk = k;
                }
            }
            if (k < kClBins) below += (double)hp[k];
        }
        if (bk > kClBins || best > mp * nb * (2.0 / 3.0)) gover[g] = 1;
        gthr[g] = bk >= kClBins ? 0xFFFFFFFFu : kClT << bk;
    }
}

// One warp per cluster: a column for a large one, its pairs for a small one.
// MB is word-major: MB[w * nm + k].  tv32 holds the tile votes as bytes
// (each below 256: at most b tables).
__global__ void __launch_bounds__(256) k_clu_apply(const unsigned long long *__restrict__ comp,
                                                   const uint64_t *__restrict__ cst, const uint64_t *__restrict__ ncl,
                                                   const uint32_t *__restrict__ mg, const DenseGroup *__restrict__ G,
                                                   uint64_t nm, uint32_t *__restrict__ gcol,
                                                   uint32_t *__restrict__ gover, uint32_t *__restrict__ MB,
                                                   uint32_t *__restrict__ tv32, const uint32_t *__restrict__ gthr) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nc = *ncl;
    for (uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; c < nc;
         c += (uint64_t)gridDim.x * blockDim.x / 32) {
        const uint64_t e0 = cst[c], e1 = cst[c + 1];
        const uint32_t sz = (uint32_t)(e1 - e0);
        if (sz < 2) continue;  // warp-uniform
        const uint32_t g = mg[comp[e0] & 0xFFFFFF];
        if (gover[g]) continue;  // voted by direct comparison
        if (sz >= gthr[g]) {
            uint32_t col = 0;
            if (lane == 0) col = atomicAdd(gcol + g, 1u);
            col = __shfl_sync(~0u, col, 0);
            if (col >= kClW * 32) {
                if (lane == 0) atomicOr(gover + g, 1u);
                continue;
            }
            for (uint64_t x = e0 + lane; x < e1; x += 32)
                atomicOr(MB + (uint64_t)(col / 32) * nm + (comp[x] & 0xFFFFFF), 1u << (col & 31));
        } else {
            const DenseGroup D = G[g];
            // pairs (a, b), a < b, of the cluster's members (ascending):
            // row a by the warp, its partners b 32 at a time
            for (uint32_t a = 0; a + 1 < sz; a++) {
                const uint32_t la = (uint32_t)(comp[e0 + a] & 0xFFFFFF) - D.g0, ta = la / kDT;
                for (uint32_t bb = a + 1 + lane; bb < sz; bb += 32) {
                    const uint32_t lb = (uint32_t)(comp[e0 + bb] & 0xFFFFFF) - D.g0;
                    const uint32_t tb = lb / kDT;
                    const uint64_t tn = D.t0 + (uint64_t)ta * D.nt - (uint64_t)ta * (ta - 1) / 2 + (tb - ta);
                    const uint64_t byte = tn * (kDT * kDT) + (la % kDT) * kDT + (lb % kDT);
                    atomicAdd(tv32 + (byte >> 2), 1u << (8 * (byte & 3)));
                }
            }
        }
    }
}

// Dense groups voted from the cluster masks: the small clusters' counts are
// already in the tile; the large ones are added as popc(mask_a & mask_b).
// Then, as k_dense_rowcount, the per-row detection counts.
__global__ void __launch_bounds__(256) k_dense_rowcount_mask(const DenseTile *__restrict__ tiles, uint64_t ntiles,
                                                             const uint32_t *__restrict__ tile_grp,
                                                             const uint32_t *__restrict__ gcol,
                                                             const uint32_t *__restrict__ gover,
                                                             const uint32_t *__restrict__ MB, uint64_t nm,
                                                             const uint32_t *__restrict__ ids, uint32_t v,
                                                             uint32_t excl, uint32_t *__restrict__ dense_cnt,
                                                             uchar4 *__restrict__ tv) {
    __shared__ __align__(16) uint32_t sA[kClW][kDT], sB[kClW][kDT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const uint32_t g = tile_grp[ti];
        if (gover[g]) continue;  // block-uniform
        const uint32_t nw = (min(gcol[g], kClW * 32) + 31) / 32;
        const DenseTile T = tiles[ti];
        const uint32_t a0 = T.g0 + T.ta * kDT, b0 = T.g0 + T.tb * kDT;
        const uint32_t na = min((uint32_t)kDT, T.n - T.ta * kDT), nbb = min((uint32_t)kDT, T.n - T.tb * kDT);
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < nw * kDT; x += blockDim.x) {
            const uint32_t w = x / kDT, c = x % kDT;
            sA[w][c] = c < na ? MB[(uint64_t)w * nm + a0 + c] : 0u;
            sB[w][c] = c < nbb ? MB[(uint64_t)w * nm + b0 + c] : 0u;
        }
        __syncthreads();
        uint32_t acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uchar4 q = tv[ti * (kDT * kDT / 4) + (ty * 4 + u) * (kDT / 4) + tx];
            acc[u][0] = q.x;
            acc[u][1] = q.y;
            acc[u][2] = q.z;
            acc[u][3] = q.w;
        }
        for (uint32_t w = 0; w < nw; w++) {
            const uint4 av = *reinterpret_cast<const uint4 *>(&sA[w][ty * 4]);
            const uint4 bv = *reinterpret_cast<const uint4 *>(&sB[w][tx * 4]);
            const uint32_t A4[4] = {av.x, av.y, av.z, av.w}, B4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[u][q] += __popc(A4[u] & B4[q]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            tv[ti * (kDT * kDT / 4) + (ty * 4 + u) * (kDT / 4) + tx] =
                make_uchar4((uint8_t)acc[u][0], (uint8_t)acc[u][1], (uint8_t)acc[u][2], (uint8_t)acc[u][3]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t ga = T.ta * kDT + ty * 4 + u;
            uint32_t c = 0;
            const uint32_t i = ga < T.n ? ids[T.g0 + ga] : 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t gb = T.tb * kDT + tx * 4 + q;
                if (ga < T.n && gb < T.n && ga < gb && acc[u][q] >= v && ids[T.g0 + gb] - i > excl) ++c;
            }
#pragma unroll
            for (int d = 8; d; d >>= 1) c += __shfl_down_sync(~0u, c, d, 16);
            if (tx == 0 && c) atomicAdd(dense_cnt + i, c);
        }
    }
}

// Dense groups, emit pass: one CTA per strip (group, row tile ta), column
// tiles taken in increasing order so every row's detections are written in
// increasing j at row_off[i] + (running count).  The votes come from the
// counting pass's tile buffer: tile (ta, tb) of a group with nt tiles per
// side is number t0 + ta*nt - ta*(ta-1)/2 + (tb - ta).
struct DenseStrip {
    uint32_t g0, n, ta, t0;
};

__global__ void __launch_bounds__(256) k_dense_rows(const DenseStrip *__restrict__ strips, uint64_t nstrips,
                                                    const uchar4 *__restrict__ tv, const uint32_t *__restrict__ ids,
                                                    uint32_t v, uint32_t excl, const uint64_t *__restrict__ row_off,
                                                    uint32_t *__restrict__ oi, uint32_t *__restrict__ oj,
                                                    uint8_t *__restrict__ ov) {
    // A tile's votes and column ids are staged in shared memory; warp w owns
    // rows 8w .. 8w + 7 of the strip: for each, two ballots give the row's
    // kept columns as a 64-bit mask and the lanes write them compacted, in
    // column order, as one coalesced run after the row's running count.
    __shared__ __align__(16) uint8_t s_v[kDT][kDT];
    __shared__ uint32_t s_rid[kDT], s_jid[kDT], s_cur[kDT];
    __shared__ uint64_t s_off[kDT];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = (1u << lane) - 1;
    for (uint64_t si = blockIdx.x; si < nstrips; si += gridDim.x) {
        const DenseStrip S = strips[si];
        const uint32_t nt = (S.n + kDT - 1) / kDT;
        __syncthreads();  // the previous strip is done with the row arrays
        if (threadIdx.x < kDT) {
            const uint32_t ga = S.ta * kDT + threadIdx.x;
            const uint32_t rid = ga < S.n ? ids[S.g0 + ga] : 0u;
            s_rid[threadIdx.x] = rid;
            s_off[threadIdx.x] = ga < S.n ? row_off[rid] : 0;
            s_cur[threadIdx.x] = 0;
        }
        const uint64_t trow = (uint64_t)S.t0 + (uint64_t)S.ta * nt - (uint64_t)S.ta * (S.ta - 1) / 2 - S.ta;
        for (uint32_t tb = S.ta; tb < nt; tb++) {
            __syncthreads();  // every warp is done with the previous tile
            const uchar4 *src = tv + (trow + tb) * (kDT * kDT / 4);
            for (uint32_t x = threadIdx.x; x < kDT * kDT / 4; x += blockDim.x)
                reinterpret_cast<uchar4 *>(&s_v[0][0])[x] = src[x];
            if (threadIdx.x < kDT) {
                const uint32_t gb = tb * kDT + threadIdx.x;
                s_jid[threadIdx.x] = gb < S.n ? ids[S.g0 + gb] : 0u;
            }
            __syncthreads();
            for (uint32_t r = warp * 8; r < warp * 8 + 8; r++) {
                const uint32_t ga = S.ta * kDT + r;
                if (ga >= S.n) break;  // warp-uniform
                const uint32_t rid = s_rid[r];
                bool keep[2];
                uint32_t m[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t col = h * 32 + lane, gb = tb * kDT + col;
                    keep[h] = gb < S.n && ga < gb && s_v[r][col] >= v && s_jid[col] - rid > excl;
                    m[h] = __ballot_sync(~0u, keep[h]);
                }
                const uint32_t cnt = __popc(m[0]) + __popc(m[1]);
                if (!cnt) continue;  // warp-uniform
                const uint64_t base = s_off[r] + s_cur[r];
#pragma unroll
                for (int h = 0; h < 2; h++)
                    if (keep[h]) {
                        const uint32_t col = h * 32 + lane;
                        const uint64_t o = base + (h ? __popc(m[0]) : 0u) + __popc(m[h] & lt);
                        oi[o] = rid;
                        oj[o] = s_jid[col];
                        ov[o] = s_v[r][col];
                    }
                __syncwarp();
                if (lane == 0) s_cur[r] += cnt;  // row r belongs to this warp alone
                __syncwarp();
            }
        }
    }
}

// Sparse detections placed after the row's dense ones; rows holding both
// kinds are listed for a merge.
__global__ void k_sparse_place(uint64_t N, const uint32_t *__restrict__ sp_cnt, const uint64_t *__restrict__ sp_start,
                               const uint32_t *__restrict__ sp_j, const uint8_t *__restrict__ sp_v,
                               const uint32_t *__restrict__ dense_cnt, const uint64_t *__restrict__ row_off,
                               uint32_t *__restrict__ oi, uint32_t *__restrict__ oj, uint8_t *__restrict__ ov,
                               uint32_t *__restrict__ merge_rows, uint64_t *__restrict__ merge_ofs,
                               unsigned long long *__restrict__ n_merge, unsigned long long *__restrict__ merge_tot) {
    // a warp takes 32 consecutive rows (coalesced counts and offsets) and
    // copies each non-empty one with all lanes (coalesced runs)
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * 32; base < N;
         base += nwarps * 32) {
        const uint64_t i = base + lane;
        uint32_t n = 0, d = 0;
        uint64_t o = 0, s = 0;
        if (i < N && (n = sp_cnt[i]) != 0) {
            d = dense_cnt ? dense_cnt[i] : 0;
            o = row_off[i] + d;
            s = sp_start[i];
        }
        for (uint32_t todo = __ballot_sync(~0u, n != 0); todo; todo &= todo - 1) {
            const int r = __ffs(todo) - 1;
            const uint32_t rn = __shfl_sync(~0u, n, r), ri = (uint32_t)(base + r);
            const uint64_t ro = __shfl_sync(~0u, o, r), rs = __shfl_sync(~0u, s, r);
            for (uint32_t k = lane; k < rn; k += 32) {
                oi[ro + k] = ri;
                oj[ro + k] = sp_j[rs + k];
                ov[ro + k] = sp_v[rs + k];
            }
        }
        if (n && d) {
            const unsigned long long q = atomicAdd(n_merge, 1ull);
            merge_rows[q] = (uint32_t)i;
            merge_ofs[q] = atomicAdd(merge_tot, (unsigned long long)(d + n));
        }
    }
}

// Rows with dense and sparse detections: the two sorted runs are merged by
// rank (each entry's position = its index in its run + entries of the other
// run with a smaller j), through scratch, one CTA per row.
__global__ void k_row_merge(const uint32_t *__restrict__ rows, uint64_t nrows, const uint32_t *__restrict__ dense_cnt,
                            const uint32_t *__restrict__ sp_cnt, const uint64_t *__restrict__ row_off,
                            uint32_t *__restrict__ oj, uint8_t *__restrict__ ov, uint32_t *__restrict__ tj,
                            uint8_t *__restrict__ tv, const uint64_t *__restrict__ tofs) {
    for (uint64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const uint32_t i = rows[r];
        const uint64_t o = row_off[i];
        const uint32_t d = dense_cnt[i], sn = sp_cnt[i];
        const uint32_t *J = oj + o;
        uint32_t *TJ = tj + tofs[r];
        uint8_t *TV = tv + tofs[r];
        for (uint32_t x = threadIdx.x; x < d + sn; x += blockDim.x) {
            const uint32_t jx = J[x];
            uint32_t lo, hi, other;
            if (x < d) lo = d, hi = d + sn, other = x;
            else lo = 0, hi = d, other = x - d;
            // entries of the other run with j < jx (binary search)
            uint32_t a = lo, b = hi;
            while (a < b) {
                uint32_t m = (a + b) / 2;
                if (J[m] < jx) a = m + 1;
                else b = m;
            }
            const uint32_t pos = other + (a - lo);
            TJ[pos] = jx;
            TV[pos] = ov[o + x];
        }
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < d + sn; x += blockDim.x) {
            oj[o + x] = TJ[x];
            ov[o + x] = TV[x];
        }
        __syncthreads();
    }
}

__global__ void k_add_u32(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, uint32_t *__restrict__ out,
                          uint64_t n) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        out[x] = a[x] + b[x];
}

// Big buckets (more than kSmall entries) of every table, and the pairs of the
// small ones (an upper bound of the sparse work).  A warp walks runs of
// 32-entry tiles with the head bitmasks of the current and next tile: a
// bucket starting at lane L ends at the next head; with no head in the two
// tiles it is big and its end is found by galloping.
// Head bitmask of tile T from its keys (one per lane) and the key before the
// tile (kprev0, position 32 T - 1; unused for T = 0).
__device__ __forceinline__ uint32_t heads_of(uint32_t key, uint32_t kprev0, const Stations &st, uint64_t N,
                                             uint64_t T) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t x = T * 32 + lane;
    const bool valid = x < N;
    uint32_t kprev = __shfl_up_sync(~0u, key, 1);
    if (lane == 0) kprev = kprev0;
    bool head = !valid || x == 0 || key != kprev;
    if (st.nst > 1 && valid && !head) head = st.soff[station_of(st, x)] == x;
    return __ballot_sync(~0u, head);
}

// Tiles are read in batches of kFB + 1 (the last one is the next batch's
// first), so a warp has kFB loads in flight instead of one.
constexpr int kFB = 8;

__global__ void __launch_bounds__(256) k_find_big(EnumArgs a, uint32_t tiles_per_warp, uint4 *__restrict__ big,
                                                  unsigned long long *__restrict__ nbig, uint64_t big_cap,
                                                  unsigned long long *__restrict__ small_pairs, uint32_t *err) {
    const uint32_t t = blockIdx.y, lane = threadIdx.x & 31;
    const uint64_t N = a.N, ntiles = (N + 31) / 32;
    const uint32_t *k = a.skey + (uint64_t)t * N;
    const uint64_t T0 = ((uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * tiles_per_warp;
    if (T0 >= ntiles) return;  // warp-uniform
    const uint64_t T1 = min(T0 + tiles_per_warp, ntiles);
    unsigned long long pairs = 0;
    uint32_t carry = T0 ? k[T0 * 32 - 1] : 0u;  // the key before the batch's first tile
    for (uint64_t B = T0; B < T1; B += kFB) {
        uint32_t kk[kFB + 1], h[kFB + 1];
#pragma unroll
        for (int u = 0; u <= kFB; u++) {
            const uint64_t x = (B + u) * 32 + lane;
            kk[u] = x < N ? __ldcs(k + x) : 0u;
        }
        uint32_t kp = carry;
#pragma unroll
        for (int u = 0; u <= kFB; u++) {
            h[u] = heads_of(kk[u], kp, a.st, N, B + u);
            kp = __shfl_sync(~0u, kk[u], 31);
        }
        carry = __shfl_sync(~0u, kk[kFB - 1], 31);
#pragma unroll
        for (int u = 0; u < kFB; u++) {
            const uint64_t T = B + u;
            if (T >= T1) break;  // warp-uniform
            const uint32_t hc = h[u], hn = h[u + 1];
            const uint64_t x = T * 32 + lane;
            if (x < N && (hc >> lane & 1)) {
                const uint64_t above = ((uint64_t)hn << 32 | hc) & ~((2ull << lane) - 1);
                const uint32_t e = above ? (uint32_t)__ffsll((long long)above) - 1 : 64u;
                const uint32_t size = e - lane;
                if (e < 64 && size <= kSmall) {
                    pairs += (unsigned long long)size * (size - 1) / 2;
                } else {
                    uint64_t hi = x + size;  // exact when the end lies in the window
                    if (e == 64) {  // gallop from the last position of the window, which is in the bucket
                        const uint64_t s1 = a.st.soff[station_of(a.st, x) + 1];
                        const uint32_t key = k[x];
                        uint64_t lo = x + size - 1, step = 1;
                        for (;;) {
                            hi = lo + step;
                            if (hi >= s1 || k[hi] != key) break;
                            lo = hi;
                            step <<= 1;
                        }
                        if (hi > s1) hi = s1;
                        while (hi - lo > 1) {
                            const uint64_t mid = lo + (hi - lo) / 2;
                            if (k[mid] == key) lo = mid;
                            else hi = mid;
                        }
                    }
                    const unsigned long long slot = atomicAdd(nbig, 1ull);
                    if (slot < big_cap) big[slot] = make_uint4(t, (uint32_t)x, (uint32_t)hi, 0);
                    else set_err(err, ERR_OVERFLOW);
                }
            }
        }
    }
    for (int o = 16; o; o >>= 1) pairs += __shfl_down_sync(~0u, pairs, o);
    if (lane == 0 && pairs) atomicAdd(small_pairs, pairs);
}

uint32_t bits_for(uint64_t N) {
    uint32_t nb = 1;
    while (nb < 32 && (1ull << nb) < N) nb++;
    return nb;
}


}  // namespace

// large_min: above the largest bucket the random background makes.  The most
// likely key of a table has probability ~(K/D)^r, so the background tops out
// near N (K/D)^r members; take 8x that, at least 512.
constexpr uint64_t kLargeRel = 16;  // dense buckets hold at least 1/16 of the largest bucket's live members

uint32_t large_min_for(const fast_ctx *c, uint64_t N) {
    if (c->large_min) return c->large_min;
    const double ptop = std::pow((double)c->p.K / c->p.D, (double)c->p.r);
    return (uint32_t)std::max(512.0, std::min(1e9, 8.0 * N * ptop));
}

// Device memory the call may still take: what the HBM budget leaves, or,
// without a budget, the device's free memory plus what the context's pool
// holds unused, less a 1 GiB margin.
uint64_t room_bytes(const fast_ctx *c) {
    if (c->budget) return c->budget > c->live ? c->budget - c->live : 0;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    uint64_t reserved = 0, used = 0;
    cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &used);
    const uint64_t avail = fr + (reserved > used ? reserved - used : 0);
    return avail > (1ull << 30) ? avail - (1ull << 30) : 0;
}

// Memory the pair buffer may take: the room less what the votes allocate
// beside it (`extra`: the slow-group list, the sparse lists, the long-row
// offsets and scratch) and a margin of 1 GiB or a sixteenth of the room;
// at most half the room when that reserve is most of it.
static uint64_t pair_room(const fast_ctx *c, uint64_t extra) {
    const uint64_t r = room_bytes(c);
    const uint64_t keep = std::max<uint64_t>(extra + (1ull << 30), r / 16);
    return r > 2 * keep ? r - keep : r / 2;
}

// Tiles of 32 table entries per warp for the warp-window passes: enough warps
// for ~16 resident per SM slot over all tables, at most 64 tiles each.
static uint32_t tiles_per_warp(const fast_ctx *c, uint64_t N, uint32_t nb) {
    const uint64_t ntiles = (N + 31) / 32;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(64, ntiles * nb / ((uint64_t)c->num_sms * 64 * 16)));
}

// ------------------------------------------------------------ host side

fast_status filter_launch(fast_ctx *c, fast_tables *tb, cudaStream_t s) {
    const fast_params &p = c->p;
    const uint64_t N = tb->N;
    fast_status st;
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
    cudaMemsetAsync(scal, 0, sizeof(uint64_t) * kScal, s);
    // big buckets of every table (the search takes the list over)
    tb->big_cap = (uint64_t)p.b * (N / (kSmall + 1) + tb->nst);
    if ((st = dalloc_t(c, &tb->d_big, tb->big_cap ? tb->big_cap : 1, s)) || (st = dalloc_t(c, &tb->d_bigcnt, 2, s)))
        return st;
    cudaMemsetAsync(tb->d_bigcnt, 0, 16, s);
    if (N) {
        EnumArgs ea{tb->d_skey, tb->d_sid, tb->d_drop, nullptr, nullptr, N, p.excl, 0, (uint32_t)N, 1,
                    {tb->d_soff, tb->nst}};
        const uint32_t ftpw = tiles_per_warp(c, N, p.b);
        const dim3 eg((unsigned)std::max<uint64_t>(1, (((N + 31) / 32 + ftpw - 1) / ftpw + 7) / 8), p.b);
        k_find_big<<<eg, 256, 0, s>>>(ea, ftpw, tb->d_big, tb->d_bigcnt, tb->big_cap, tb->d_bigcnt + 1, c->d_err),
            FAST_LAUNCHED(c);
    }
    uint32_t *heavy = nullptr;
    if (p.occ_num > 0 && N > 0) {
        uint64_t smin = ~0ull;  // smallest heavy size over the stations
        for (uint32_t x = 0; x < tb->nst; x++)
            if (tb->soff[x + 1] > tb->soff[x])
                smin = std::min<uint64_t>(smin, (uint64_t)p.occ_num * (tb->soff[x + 1] - tb->soff[x]) / p.occ_den + 1);
        if ((st = dalloc_t(c, &heavy, N, s))) return st;
        cudaMemsetAsync(heavy, 0, N * 4, s);
        if (smin > kSmall) {  // every heavy bucket is a big one
            k_heavy_mark<<<c->num_sms * 4, 256, 0, s>>>(tb->d_big, tb->d_bigcnt, tb->big_cap,
                                                        Stations{tb->d_soff, tb->nst}, p.occ_num, p.occ_den, tb->d_sid,
                                                        N, heavy), FAST_LAUNCHED(c);
        } else {  // small stations: heavy buckets among the small ones too, found by a scan
            const uint64_t cap = (uint64_t)p.b * (N / smin + tb->nst);
            if (cap > (1ull << 26)) return set_error(c, FAST_EBUDGET, "occurrence threshold too small for this N");
            uint4 *list = nullptr;
            if ((st = dalloc_t(c, &list, cap, s))) return st;
            dim3 g(std::max(1u, std::min<unsigned>(ceil_div(N, 256), 4096)), p.b);
            k_heavy_find<<<g, 256, 0, s>>>(tb->d_skey, N, Stations{tb->d_soff, tb->nst}, p.occ_num, p.occ_den, list,
                                           scal + Scal::NHEAVY, cap, c->d_err), FAST_LAUNCHED(c);
            k_heavy_mark_list<<<c->num_sms * 4, 256, 0, s>>>(list, scal + Scal::NHEAVY, cap, tb->d_sid, N, heavy),
                FAST_LAUNCHED(c);
            dfree(c, list, cap * sizeof(uint4), s);
        }
    }
    k_drop<<<std::max(1u, std::min<unsigned>(ceil_div(N, 256), c->num_sms * 8)), 256, 0, s>>>(heavy, N, p.b, tb->d_drop,
                                                                                             scal + Scal::NDROP), FAST_LAUNCHED(c);
    if (heavy) dfree(c, heavy, N * 4, s);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(c, e, "filter");
    if (c->capturing) return FAST_OK;  // the plan reads the counters after the graph runs
    cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(uint64_t) * kScal, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "occurrence filter"))) return st;
    tb->n_dropped = c->h_scal[Scal::NDROP];
    return FAST_OK;
}

static fast_status read_scal(fast_ctx *c, cudaStream_t s, const char *where) {
    cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(uint64_t) * kScal, cudaMemcpyDeviceToHost, s);
    return sync_check(c, s, where);
}

// Global-map search: sparse pairs summed in one open-addressing hash map of
// packed (i, j) -> votes per query partition, output ordered by a radix sort.
static fast_status search_map(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, fast_result **out,
                              cudaStream_t s) {
    const fast_params &p = c->p;
    const uint64_t N = tb->N;
    const uint32_t nb = p.b;
    const uint32_t nbits = bits_for(N);
    fast_status st = FAST_OK;
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
    std::vector<std::pair<void *, size_t>> owned;  // freed at the end
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
    auto fail = [&](fast_status r) {
        release();
        return r;
    };

    c->stats.n_fingerprints = N;
    c->stats.n_dropped = tb->n_dropped;

    const uint32_t large_min = large_min_for(c, N);

    uint32_t nparts = p.query_part ? p.query_part : 1;
    nparts = std::min<uint32_t>(nparts, 64);

    // ---- pass 1: big buckets and small-pair counts
    stage_mark(c, 3, s);
    cudaMemsetAsync(scal, 0, sizeof(uint64_t) * kScal, s);
    const uint64_t big_cap = (uint64_t)nb * (N / (kSmall + 1) + 1);
    uint4 *big = nullptr, *large = nullptr, *medium = nullptr;
    if ((st = alloc(&big, big_cap))) return fail(st);
    EnumArgs ea{tb->d_skey, tb->d_sid, tb->d_drop, nullptr, nullptr, N, p.excl, 0, (uint32_t)N, nparts, {tb->d_soff, tb->nst}};
    Map nomap{nullptr, 0};
    const dim3 eg(std::max(1u, std::min<unsigned>(ceil_div(N, 256), 2048)), nb);
    k_enum<0><<<eg, 256, 0, s>>>(ea, big, scal + Scal::NBIG, big_cap, scal + Scal::PART0, nomap, c->d_err), FAST_LAUNCHED(c);
    if ((st = read_scal(c, s, "bucket scan"))) return fail(st);
    const uint64_t nbig = c->h_scal[Scal::NBIG];
    if ((st = alloc(&large, nbig)) || (st = alloc(&medium, nbig))) return fail(st);
    k_big_classify<<<std::max<uint64_t>(1, std::min<uint64_t>(nbig, c->num_sms * 8)), 256, 0, s>>>(
        ea, big, scal + Scal::NBIG, big_cap, large_min, large, scal + Scal::NLARGE, medium, scal + Scal::NMEDIUM,
        scal + Scal::PART0), FAST_LAUNCHED(c);
    if ((st = read_scal(c, s, "bucket classify"))) return fail(st);
    const uint64_t nlarge = c->h_scal[Scal::NLARGE], nmedium = c->h_scal[Scal::NMEDIUM];
    std::vector<uint64_t> part_ub(nparts);
    uint64_t sparse_ub = 0;
    for (uint32_t q = 0; q < nparts; q++) sparse_ub += (part_ub[q] = c->h_scal[Scal::PART0 + q]);
    stage_mark(c, 4, s);

    // ---- dense groups
    uint32_t *label = nullptr;
    uint64_t nm = 0, dense_pairs = 0, ngroups = 0, M_dense = 0;
    uint32_t *GT = nullptr, *ids = nullptr;
    std::vector<DenseTile> tiles;
    DenseTile *d_tiles = nullptr;
    if ((st = alloc(&label, N))) return fail(st);
    cudaMemsetAsync(label, 0xFF, N * 4, s);
    if (nlarge) {
        const unsigned lg = (unsigned)std::min<uint64_t>(nlarge, c->num_sms * 8);
        k_label_init<<<lg, 256, 0, s>>>(large, nlarge, tb->d_sid, tb->d_drop, N, label), FAST_LAUNCHED(c);
        int it = 0;
        for (; it < 256; it++) {
            cudaMemsetAsync(scal + Scal::CHANGED, 0, 8, s);
            k_label_prop<<<lg, 256, 0, s>>>(large, nlarge, tb->d_sid, tb->d_drop, N, label,
                                            reinterpret_cast<uint32_t *>(scal + Scal::CHANGED)), FAST_LAUNCHED(c);
            if ((st = read_scal(c, s, "group labels"))) return fail(st);
            if (!c->h_scal[Scal::CHANGED]) break;
        }
        if (it == 256) return fail(set_error(c, FAST_EINTERNAL, "group labels did not converge"));
        // members sorted by (label, id)
        cudaMemsetAsync(scal + Scal::NMEMB, 0, 8, s);
        unsigned long long *memb = nullptr, *memb2 = nullptr;
        if ((st = alloc(&memb, N))) return fail(st);
        k_collect_members<<<std::max(1u, std::min<unsigned>(ceil_div(N, 256), c->num_sms * 8)), 256, 0, s>>>(
            label, N, memb, scal + Scal::NMEMB), FAST_LAUNCHED(c);
        if ((st = read_scal(c, s, "group members"))) return fail(st);
        nm = c->h_scal[Scal::NMEMB];
        if ((st = alloc(&memb2, nm))) return fail(st);
        uint64_t *sorted = nullptr;
        if ((st = sort_u64(c, nm, reinterpret_cast<uint64_t *>(memb), reinterpret_cast<uint64_t *>(memb2), 0,
                           32 + nbits, &sorted, s)))
            return fail(st);
        std::vector<uint64_t> hm(nm);
        cudaMemcpyAsync(hm.data(), sorted, nm * 8, cudaMemcpyDeviceToHost, s);
        if ((st = sync_check(c, s, "group members copy"))) return fail(st);
        if ((st = alloc(&GT, (size_t)nm * nb)) || (st = alloc(&ids, nm))) return fail(st);
        k_gather_keys<<<std::max(1u, std::min<unsigned>(ceil_div(nm, 128), c->num_sms * 8)), 128, 0, s>>>(
            reinterpret_cast<unsigned long long *>(sorted), nm, d_sig, N, nb, GT, ids), FAST_LAUNCHED(c);
        // group segments and the tile schedule
        uint64_t g0 = 0;
        while (g0 < nm) {
            uint64_t g1 = g0 + 1;
            while (g1 < nm && (hm[g1] >> 32) == (hm[g0] >> 32)) g1++;
            const uint32_t n = (uint32_t)(g1 - g0);
            ngroups++;
            dense_pairs += (uint64_t)n * (n - 1) / 2;
            const uint32_t nt = (n + kDT - 1) / kDT;
            for (uint32_t a = 0; a < nt; a++)
                for (uint32_t b = a; b < nt; b++) tiles.push_back({(uint32_t)g0, n, a, b});
            g0 = g1;
        }
        if ((st = alloc(&d_tiles, tiles.size()))) return fail(st);
        cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(DenseTile), cudaMemcpyHostToDevice, s);
        const size_t dsm = (size_t)2 * nb * kDT * 4;
        cudaFuncSetAttribute(k_dense<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        cudaFuncSetAttribute(k_dense<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        const unsigned dg = (unsigned)std::min<uint64_t>(tiles.size(), (uint64_t)c->num_sms * 4);
        cudaMemsetAsync(scal + Scal::CUR_DENSE, 0, 8, s);
        k_dense<0><<<dg, 256, dsm, s>>>(d_tiles, tiles.size(), GT, ids, nm, nb, p.v, p.excl, nbits, nullptr,
                                        scal + Scal::CUR_DENSE, 0, c->d_err), FAST_LAUNCHED(c);
        if ((st = read_scal(c, s, "dense count"))) return fail(st);
        M_dense = c->h_scal[Scal::CUR_DENSE];
    }

    // ---- sparse vote map, one query partition at a time
    uint64_t M_cap = M_dense;
    // sparse detections need >= v emissions each
    M_cap += sparse_ub / std::max<uint32_t>(1, p.v) + 1;
    unsigned long long *outk = nullptr, *outk2 = nullptr;
    if ((st = alloc(&outk, M_cap))) return fail(st);
    cudaMemsetAsync(scal + Scal::CUR_DENSE, 0, 8, s);
    if (nlarge && M_dense) {
        const size_t dsm = (size_t)2 * nb * kDT * 4;
        const unsigned dg = (unsigned)std::min<uint64_t>(tiles.size(), (uint64_t)c->num_sms * 4);
        k_dense<1><<<dg, 256, dsm, s>>>(d_tiles, tiles.size(), GT, ids, nm, nb, p.v, p.excl, nbits, outk,
                                        scal + Scal::CUR_DENSE, M_cap, c->d_err), FAST_LAUNCHED(c);
    }
    stage_mark(c, 5, s);
    ea.label = label;
    uint64_t max_part = *std::max_element(part_ub.begin(), part_ub.end());
    const uint64_t map_cap = std::max<uint64_t>(1024, (uint64_t)((double)max_part / c->map_load) + 1);
    unsigned long long *slots = nullptr;
    if ((st = alloc(&slots, map_cap))) return fail(st);
    cudaMemsetAsync(scal + Scal::CUR_SPARSE, 0, 8, s);
    for (uint32_t q = 0; q < nparts; q++) {
        if (part_ub[q] == 0) continue;
        const uint64_t cap_q = std::max<uint64_t>(1024, (uint64_t)((double)part_ub[q] / c->map_load) + 1);
        cudaMemsetAsync(slots, 0, cap_q * 8, s);
        Map m{slots, cap_q};
        ea.i_lo = (uint32_t)((uint64_t)q * N / nparts);
        ea.i_hi = (uint32_t)((uint64_t)(q + 1) * N / nparts);
        // ceil so that i * nparts / N == q exactly on [i_lo, i_hi)
        ea.i_lo = (uint32_t)(((uint64_t)q * N + nparts - 1) / nparts);
        ea.i_hi = (uint32_t)(((uint64_t)(q + 1) * N + nparts - 1) / nparts);
        k_enum<1><<<eg, 256, 0, s>>>(ea, nullptr, nullptr, 0, nullptr, m, c->d_err), FAST_LAUNCHED(c);
        if (nmedium) {
            k_medium<<<(unsigned)std::min<uint64_t>(nmedium, c->num_sms * 8), 256, 0, s>>>(
                ea, medium, scal + Scal::NMEDIUM, m, c->d_err), FAST_LAUNCHED(c);
        }
        const unsigned cg = (unsigned)std::min<uint64_t>(ceil_div(cap_q, 256), c->num_sms * 16);
        k_map_compact<1><<<cg, 256, 0, s>>>(slots, cap_q, p.v, nbits, outk + M_dense, scal + Scal::CUR_SPARSE,
                                            M_cap - M_dense, c->d_err), FAST_LAUNCHED(c);
    }
    c->stats.map_slots = map_cap;
    if ((st = read_scal(c, s, "sparse votes"))) return fail(st);
    const uint64_t M_sparse = c->h_scal[Scal::CUR_SPARSE];
    stage_mark(c, 6, s);

    // ---- canonical order and unpack
    const uint64_t M = M_dense + M_sparse;
    if ((st = alloc(&outk2, M))) return fail(st);
    uint64_t *sorted = reinterpret_cast<uint64_t *>(outk);
    if (M > 1 &&
        (st = sort_u64(c, M, reinterpret_cast<uint64_t *>(outk), reinterpret_cast<uint64_t *>(outk2), 8, 8 + 2 * nbits,
                       &sorted, s)))
        return fail(st);
    fast_result *res = new fast_result();
    res->ctx = c;
    res->stream = s;
    res->M = M;
    if ((st = dalloc_t(c, &res->d_i, M ? M : 1, s)) || (st = dalloc_t(c, &res->d_j, M ? M : 1, s)) ||
        (st = dalloc_t(c, &res->d_votes, M ? M : 1, s))) {
        fast_result_free(res);
        return fail(st);
    }
    if (M)
        k_unpack<<<std::max(1u, std::min<unsigned>(ceil_div(M, 256), c->num_sms * 16)), 256, 0, s>>>(
            reinterpret_cast<unsigned long long *>(sorted), M, nbits, res->d_i, res->d_j, res->d_votes), FAST_LAUNCHED(c);
    release();
    stage_mark(c, 8, s);
    if ((st = sync_check(c, s, "search output"))) {
        fast_result_free(res);
        return st;
    }
    c->stats.n_emissions = sparse_ub;
    c->stats.n_dense_pairs = dense_pairs;
    c->stats.n_groups = ngroups;
    c->stats.n_detections = M;
    c->stats.query_parts = nparts;
    *out = res;
    return FAST_OK;
}


// Sparse pairs of small and medium buckets: count per group, scan, append,
// vote per row.  PT is the packed entry type (local row, j).
// First position of each group in the overflow list of a single-pass
// emission (sorted by group).
__global__ void k_ovf_starts(const unsigned long long *__restrict__ ovf, uint64_t n, uint64_t *__restrict__ ostart) {
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t g = ovf[q] >> 32;
        if (q == 0 || (ovf[q - 1] >> 32) != g) ostart[g] = q;
    }
}

// cut[2q] = first row group whose pair offset reaches q/nparts of all S
// pairs, cut[2q + 1] = that group's offset (q = 0 .. nparts)
__global__ void k_part_cuts(const uint64_t *__restrict__ goff, uint64_t ng, uint64_t S, uint32_t nparts,
                            uint64_t *__restrict__ cut) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > nparts) return;
    const uint64_t want = (uint64_t)((unsigned __int128)S * q / nparts);
    uint64_t lo = 0, hi = ng + 1;  // first g with goff[g] >= want
    while (lo < hi) {
        const uint64_t m = (lo + hi) / 2;
        if (goff[m] < want) lo = m + 1;
        else hi = m;
    }
    const uint64_t g = min(lo, ng);
    cut[2 * q] = g;
    cut[2 * q + 1] = goff[g];
}

// The medium-bucket writers of one pass: the warp kernel over the small
// buckets, then the CTA kernel over the rest (persistent grids: every
// resident CTA takes work until the lists are done).
template <int MODE, typename PT>
static void medium_launch(fast_ctx *c, const EnumArgs &ea, const MedLists &ml, uint32_t large_min, uint32_t gshift,
                          uint32_t nbits, uint32_t *gcnt, unsigned long long *gpos, uint32_t *gcur, PT *ent,
                          GroupRange gr, RegionSink rs, cudaStream_t s) {
    static int occ_w = 0, occ_c = 0;
    const size_t csm = (size_t)2 * kMedCap * 4;
    cudaFuncSetAttribute(k_medium_grp<MODE, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * kMedHugeCap * 4));
    if (!occ_w) {  // occupancies are the same on every device of this architecture
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_medium_warp<MODE, PT>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k_medium_grp<MODE, PT>, 256, csm);
        occ_w = std::max(occ_w, 1);
        occ_c = std::max(occ_c, 1);
    }
    k_medium_warp<MODE, PT><<<c->num_sms * occ_w, 256, 0, s>>>(ea, ml, gshift, nbits, gcnt, gpos, gcur, ent, gr,
                                                                 rs), FAST_LAUNCHED(c);
    if (large_min > kMedCap + 1) {  // live members of a medium bucket stay below large_min
        const uint32_t hcap = std::min(large_min, kMedHugeCap);
        const size_t hsm = (size_t)2 * hcap * 4;
        int occ_h = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_h, k_medium_grp<MODE, PT>, 256, hsm);
        cudaMemsetAsync(ml.next_h, 0, 8, s);
        k_medium_grp<MODE, PT><<<c->num_sms * std::max(occ_h, 1), 256, hsm, s>>>(
            ea, ml, true, hcap, gshift, nbits, gcnt, gpos, gcur, ent, gr, rs), FAST_LAUNCHED(c);
    }
    cudaMemsetAsync(ml.next, 0, 8, s);
    k_medium_grp<MODE, PT><<<c->num_sms * occ_c, 256, csm, s>>>(ea, ml, false, kMedCap, gshift, nbits, gcnt, gpos,
                                                                  gcur, ent, gr, rs), FAST_LAUNCHED(c);
}

template <typename PT, typename Alloc>
static fast_status sparse_groups(fast_ctx *c, const EnumArgs &ea, const uint4 *medium, uint64_t nmedium,
                                 uint32_t large_min, double dens, uint32_t gshift, uint32_t nbits, uint32_t *sp_cnt, uint64_t *sp_start,
                                 uint32_t **sp_j_out, uint8_t **sp_v_out, uint64_t *sp_n_out, uint2 *long_rows,
                                 uint64_t &S_out, Alloc &alloc, cudaStream_t s, uint64_t S_ub) {
    const fast_params &p = c->p;
    const uint64_t N = ea.N;
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
    fast_status st;
    const uint64_t ng = (N + (1ull << gshift) - 1) >> gshift;
    // what the votes allocate beside the pair buffer: slow-group list, long-row
    // offsets, first sparse lists, long-row scratch (at most 2 GiB per launch)
    const uint64_t vote_extra = 8 * ng + 8 * N + 5 * std::max<uint64_t>(N, 1 << 20) + (2ull << 30);
    c->stats.ms_k_pairs = c->stats.ms_k_medium = c->stats.ms_k_vote = c->stats.ms_k_vote_block = 0.f;
    c->stats.ms_k_count_small = c->stats.ms_k_count_medium = 0.f;
    // the pair buffers live only as long as this function: they are given
    // back before the detection list is allocated
    std::vector<std::pair<void *, size_t>> local;
    struct Freer {
        fast_ctx *c;
        cudaStream_t s;
        std::vector<std::pair<void *, size_t>> &v;
        ~Freer() {
            for (auto &x : v) dfree(c, x.first, x.second, s);
        }
    } freer{c, s, local};
    auto lalloc = [&](auto **ptr, size_t count) -> fast_status {
        using T = std::remove_reference_t<decltype(**ptr)>;
        fast_status r = dalloc_t(c, ptr, count ? count : 1, s);
        if (!r) local.push_back({(void *)*ptr, (count ? count : 1) * sizeof(T)});
        return r;
    };
    uint32_t *gcnt = nullptr, *gcur = nullptr;
    uint64_t *goff = nullptr;
    PT *ent = nullptr;
    if ((st = lalloc(&gcnt, ng)) || (st = lalloc(&gcur, ng)) || (st = lalloc(&goff, ng + 1))) return st;
    cudaMemsetAsync(gcnt, 0, ng * 4, s);
    cudaMemsetAsync(gcur, 0, ng * 4, s);
    // small-bucket pairs: warps over runs of 32-entry tiles
    const uint64_t ntiles = (N + 31) / 32;
    const uint32_t tpw = tiles_per_warp(c, N, p.b);
    const uint64_t nwarps = (ntiles + tpw - 1) / tpw;
    const dim3 eg((unsigned)std::max<uint64_t>(1, (nwarps + 7) / 8), p.b);
    // medium buckets: the warp list and the CTA list (largest first)
    // (counted first, then allocated at their sizes)
    uint4 *med_w = nullptr, *med_c = nullptr, *med_h = nullptr;
    uint64_t n_cta = 0;
    const unsigned sg = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(nmedium, 256), c->num_sms * 8));
    cudaMemsetAsync(scal + Scal::NMEDW, 0, 8 * 4, s);
    if (nmedium) {
        k_med_split<<<sg, 256, 0, s>>>(medium, scal + Scal::NMEDIUM, nullptr, scal + Scal::NMEDW, nullptr, 0,
                                       scal + Scal::NMEDF, scal + Scal::NMEDB, nullptr, scal + Scal::NMEDH, true),
            FAST_LAUNCHED(c);
        cudaMemcpyAsync(c->h_scal + Scal::NMEDW, scal + Scal::NMEDW, 8 * 4, cudaMemcpyDeviceToHost, s);
        if ((st = sync_check(c, s, "medium classes"))) return st;
        n_cta = c->h_scal[Scal::NMEDF] + c->h_scal[Scal::NMEDB];
        if ((st = lalloc(&med_w, c->h_scal[Scal::NMEDW])) || (st = lalloc(&med_c, n_cta)) ||
            (st = lalloc(&med_h, c->h_scal[Scal::NMEDH])))
            return st;
        cudaMemsetAsync(scal + Scal::NMEDW, 0, 8 * 4, s);
        k_med_split<<<sg, 256, 0, s>>>(medium, scal + Scal::NMEDIUM, med_w, scal + Scal::NMEDW, med_c, n_cta,
                                       scal + Scal::NMEDF, scal + Scal::NMEDB, med_h, scal + Scal::NMEDH, false),
            FAST_LAUNCHED(c);
    }
    const MedLists ml{med_w, med_c, med_h, scal + Scal::NMEDW, scal + Scal::NMEDF, scal + Scal::NMEDB,
                      scal + Scal::NMEDH, n_cta, scal + Scal::MEDNEXT, scal + Scal::MEDNEXTH};
    cudaMemsetAsync(scal + Scal::NSMALLEMIT, 0, 8, s);
    const GroupRange all{0, ng, 0};
    uint64_t S = 0;
    // Single pass (one row partition, 32-bit entries, room for regions of
    // about twice the expected group size): pairs are written once into
    // fixed group regions and compacted; otherwise counted, then written.
    bool single = false;
    c->stats.n_overflow = 0;
    uint32_t rcap = 0;
    const unsigned long long *ovf_sorted = nullptr;
    uint64_t *ostart = nullptr;
    c->stats.group_shift = gshift;
    if (sizeof(PT) == 4 && p.query_part <= 1 && c->single_pass) {
        // 2.5, 2 or 1.75 times the expected group size of the densest
        // station (`dens` times the mean; the most that fits) in whole
        // 128-byte lines -- not the power of two above twice the mean, which
        // jumps from 2x to 4x the mean as the mean crosses a power of two --
        // plus one line so that region starts do not all fall on the same
        // DRAM channels
        const uint64_t ovf_cap = c->group_slots ? S_ub + (1 << 20) : std::max<uint64_t>(1 << 20, S_ub / 8);
        const uint64_t room = pair_room(c, vote_extra);
        uint32_t cap = 0;
        for (const uint64_t quarters : {10u, 8u, 7u}) {
            const uint64_t want = ((uint64_t)(dens * quarters * (S_ub / ng + 1)) / 4 + 31) / 32 * 32;
            cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(want, 256), 1u << 16) + 32;
            if (c->group_slots) cap = c->group_slots;
            if (ng * cap * 4 + ovf_cap * 16 <= room) break;
        }
        const uint64_t need = ng * cap * 4 + ovf_cap * 16;
        uint32_t *region = nullptr;
        unsigned long long *ovf = nullptr;
        if (need <= room && !(st = lalloc(&region, ng * cap)) && !(st = lalloc(&ovf, ovf_cap))) {
            EnumArgs e1 = ea;  // ids flagged from the bitmap, no flagged copy
            e1.fsid = nullptr;
            e1.fsid_out = nullptr;
            const RegionSink rs{region, cap, ovf, ovf_cap, scal + Scal::NOVF};
            cudaMemsetAsync(scal + Scal::NOVF, 0, 8, s);
            stage_mark(c, 10, s);
            k_pairs_grp<2, PT><<<eg, 256, 0, s>>>(e1, gshift, nbits, tpw, nullptr, nullptr, gcur, nullptr,
                                                  scal + Scal::NSMALLEMIT, all, rs), FAST_LAUNCHED(c);
            stage_mark(c, 12, s);
            if (nmedium)
                medium_launch<2, PT>(c, e1, ml, large_min, gshift, nbits, nullptr, nullptr, gcur, nullptr, all, rs, s);
            stage_mark(c, 19, s);
            if ((st = scan_excl(c, gcur, goff, ng, 1, goff + ng, s))) return st;
            cudaMemcpyAsync(&S, goff + ng, 8, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(c->h_scal + Scal::NSMALLEMIT, scal + Scal::NSMALLEMIT, 8, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(c->h_scal + Scal::NOVF, scal + Scal::NOVF, 8, cudaMemcpyDeviceToHost, s);
            if ((st = sync_check(c, s, "pair pass"))) return st;
            c->stats.ms_k_pairs += stage_ms(c, 10, 12);
            c->stats.ms_k_medium += stage_ms(c, 12, 19);
            const uint64_t novf = c->h_scal[Scal::NOVF];
            c->stats.n_overflow = novf;
            if (novf <= ovf_cap) {  // the vote reads the regions and the sorted overflow list in place
                single = true;
                c->stats.region_slots = cap;
                ent = reinterpret_cast<PT *>(region);
                rcap = cap;
                if (novf) {
                    unsigned long long *ovf2 = nullptr;
                    uint64_t *srt = nullptr;
                    if ((st = lalloc(&ovf2, novf)) || (st = lalloc(&ostart, ng))) return st;
                    if ((st = sort_u64(c, novf, reinterpret_cast<uint64_t *>(ovf), reinterpret_cast<uint64_t *>(ovf2),
                                       32, 32 + bits_for(ng), &srt, s)))
                        return st;
                    ovf_sorted = reinterpret_cast<const unsigned long long *>(srt);
                    k_ovf_starts<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(novf, 256),
                                                                                        c->num_sms * 8)),
                                   256, 0, s>>>(ovf_sorted, novf, ostart), FAST_LAUNCHED(c);
                }
                stage_mark(c, 11, s);
            } else {  // overflow list too short: count, then write
                cudaMemsetAsync(gcur, 0, ng * 4, s);
                cudaMemsetAsync(scal + Scal::NSMALLEMIT, 0, 8, s);
            }
        }
        if (st) {  // the regions did not fit the device: count, then write (not an error of the call)
            st = FAST_OK;
            c->err.clear();
        }
    }
    if (!single) {
        stage_mark(c, 16, s);
        k_pairs_grp<0, PT><<<eg, 256, 0, s>>>(ea, gshift, nbits, tpw, gcnt, nullptr, nullptr, nullptr,
                                              scal + Scal::NSMALLEMIT, all), FAST_LAUNCHED(c);
        stage_mark(c, 17, s);
        if (nmedium)
            medium_launch<0, PT>(c, ea, ml, large_min, gshift, nbits, gcnt, nullptr, nullptr, nullptr, all, RegionSink{}, s);
        stage_mark(c, 18, s);
        if ((st = scan_excl(c, gcnt, goff, ng, 1, goff + ng, s))) return st;
        cudaMemcpyAsync(&S, goff + ng, 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(c->h_scal + Scal::NSMALLEMIT, scal + Scal::NSMALLEMIT, 8, cudaMemcpyDeviceToHost, s);
        if ((st = sync_check(c, s, "pair count"))) return st;
        c->stats.ms_k_count_small = stage_ms(c, 16, 17);
        c->stats.ms_k_count_medium = stage_ms(c, 17, 18);
    }
    S_out = S;
    c->stats.n_pairs_small = c->h_scal[Scal::NSMALLEMIT];
    unsigned long long *gpos = nullptr;  // the counted pass's group cursors
    if (!single && (st = lalloc(&gpos, ng))) return st;

    // Query partitions (§6.4): consecutive row-group ranges of about equal
    // pair counts, each written and voted in turn, so the pair buffer holds
    // one range.  As many as query_part asks for, or as the HBM budget needs.
    uint32_t nparts = std::max<uint32_t>(1, p.query_part);
    if (!single) {
        const uint64_t room = pair_room(c, vote_extra);
        const uint64_t need = S * sizeof(PT);
        if (room && need > room) nparts = std::max<uint64_t>(nparts, (need + room - 1) / room);
    }
    nparts = (uint32_t)std::min<uint64_t>(nparts, std::max<uint64_t>(1, ng));
    std::vector<uint64_t> cut{0, ng}, hgb{0, S};  // group boundaries of the partitions, goff there
    uint64_t part_max = S;
    uint64_t *d_cut = nullptr;
    if ((st = lalloc(&d_cut, 2 * (4096 + 1)))) return st;
    for (;;) {
        if (nparts > 1) {  // cuts of about equal pair counts, found on the device
            k_part_cuts<<<ceil_div(nparts + 1, 128), 128, 0, s>>>(goff, ng, S, nparts, d_cut), FAST_LAUNCHED(c);
            std::vector<uint64_t> hc(2 * (nparts + 1));
            cudaMemcpyAsync(hc.data(), d_cut, hc.size() * 8, cudaMemcpyDeviceToHost, s);
            if ((st = sync_check(c, s, "partition cuts"))) return st;
            cut.assign(1, 0);
            hgb.assign(1, 0);
            for (uint32_t q = 1; q < nparts; q++)
                if (hc[2 * q] > cut.back() && hc[2 * q] < ng) {
                    cut.push_back(hc[2 * q]);
                    hgb.push_back(hc[2 * q + 1]);
                }
            cut.push_back(ng);
            hgb.push_back(S);
            part_max = 0;
            for (size_t q = 0; q + 1 < cut.size(); q++) part_max = std::max(part_max, hgb[q + 1] - hgb[q]);
        }
        if (single || !(st = lalloc(&ent, part_max))) break;
        // the buffer did not fit after all (the pool's free memory can be
        // fragmented): twice the partitions
        if ((st != FAST_ENOMEM && st != FAST_EBUDGET) || nparts >= std::min<uint64_t>(ng, 4096)) return st;
        st = FAST_OK;
        c->err.clear();
        nparts = (uint32_t)std::min<uint64_t>(std::min<uint64_t>(ng, 4096), 2ull * nparts);
    }
    c->stats.query_parts = (uint32_t)(cut.size() - 1);

    // hash capacity: twice the power of two above the target (group sizes vary), at least 4096
    uint32_t vcap = 64;
    while (vcap < (c->group_pairs ? c->group_pairs : kVTargetDefault)) vcap <<= 1;
    vcap = std::min<uint32_t>(std::max<uint32_t>(2 * vcap, 4096), sizeof(PT) == 4 ? 1u << 14 : 1u << 13);
    const size_t vsm = group_vote_smem<PT>(vcap);
    cudaFuncSetAttribute(k_group_vote<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm);
    int vper = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&vper, k_group_vote<PT>, 256, vsm);
    const size_t wsm = warp_vote_smem<PT>();
    cudaFuncSetAttribute(k_warp_vote<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
    int wper = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, k_warp_vote<PT>, kVW * 32, wsm);
    uint2 *slow = nullptr;  // (group, rows r0 << 16 | r1) left to the block kernel
    if ((st = lalloc(&slow, 8 * ng))) return st;
    // long rows' offsets into their global hash scratch (one list for every
    // partition); the scratch itself is allocated at the first need
    uint64_t *d_gofs = nullptr;
    if ((st = lalloc(&d_gofs, N))) return st;
    uint32_t *gscr = nullptr;
    uint64_t gscr_cap = 0;
    struct Scratch {
        fast_ctx *c;
        cudaStream_t s;
        uint32_t *&p;
        uint64_t &n;
        ~Scratch() {
            if (p) dfree(c, p, n * 4, s);
        }
    } gscr_guard{c, s, gscr, gscr_cap};
    const size_t rsm = (size_t)2 * kRowBlockSlots * 4;
    cudaFuncSetAttribute(k_long_vote<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    uint64_t sp_cap = std::max<uint64_t>(N, 1 << 20);
    VoteArgs va{goff, ng, N, 0, ng, 0, gshift, nbits, p.v, vcap, sp_cnt, sp_start, nullptr, nullptr, 0,
                scal + Scal::CUR_SPARSE, long_rows, scal + Scal::NLONG, N,
                single ? gcur : nullptr, rcap, ovf_sorted, ostart};
    // the sparse detection lists outlive this function (the caller places
    // them); a second attempt with their exact size first gives back the
    // first attempt's, too short ones
    struct SpLists {
        fast_ctx *c;
        cudaStream_t s;
        uint32_t *j = nullptr;
        uint8_t *v = nullptr;
        uint64_t n = 0;
        bool keep = false;
        void drop() {
            if (j) dfree(c, j, n * 4, s);
            if (v) dfree(c, v, n, s);
            j = nullptr;
            v = nullptr;
            n = 0;
        }
        ~SpLists() {
            if (!keep) drop();
        }
    } sp{c, s};
    for (int attempt = 0; attempt < 2; attempt++) {
        sp.drop();
        if ((st = dalloc_t(c, &sp.j, sp_cap, s)) || (st = dalloc_t(c, &sp.v, sp_cap, s))) return st;
        sp.n = sp_cap;
        va.sp_j = sp.j;
        va.sp_v = sp.v;
        va.sp_cap = sp_cap;
        cudaMemsetAsync(sp_cnt, 0, N * 4, s);
        cudaMemsetAsync(scal + Scal::CUR_SPARSE, 0, 8, s);
        c->stats.n_long_rows = c->stats.n_huge_rows = 0;
        for (size_t q = 0; q + 1 < cut.size(); q++) {
            const GroupRange gr{cut[q], cut[q + 1], cut.size() > 2 ? hgb[q] : 0};
            va.g_lo = gr.g_lo;
            va.g_hi = gr.g_hi;
            va.ebase = gr.ebase;
            // write the range's pairs (each group's cursor starts at its offset in the range's buffer)
            if (!single) {
                k_init_pos<<<(unsigned)std::max<uint64_t>(
                                 1, std::min<uint64_t>(ceil_div(gr.g_hi - gr.g_lo, 256), c->num_sms * 8)),
                             256, 0, s>>>(goff, gr, gpos), FAST_LAUNCHED(c);
                stage_mark(c, 10, s);
                k_pairs_grp<1, PT><<<eg, 256, 0, s>>>(ea, gshift, nbits, tpw, nullptr, gpos, gcur, ent, nullptr, gr),
                    FAST_LAUNCHED(c);
                stage_mark(c, 12, s);
                if (nmedium)
                    medium_launch<1, PT>(c, ea, ml, large_min, gshift, nbits, nullptr, gpos, gcur, ent, gr,
                                         RegionSink{}, s);
                stage_mark(c, 11, s);
            }
            // vote the range
            cudaMemsetAsync(scal + Scal::NLONG, 0, 8, s);
            cudaMemsetAsync(scal + Scal::NSLOW, 0, 8, s);
            stage_mark(c, 13, s);
            const uint64_t ngr = gr.g_hi - gr.g_lo;
            k_warp_vote<PT><<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>((ngr + kVW - 1) / kVW,
                                                                                  (uint64_t)c->num_sms *
                                                                                      std::max(wper, 1))),
                              kVW * 32, wsm, s>>>(va, ent, slow, scal + Scal::NSLOW), FAST_LAUNCHED(c);
            stage_mark(c, 14, s);
            k_group_vote<PT><<<(unsigned)std::max<uint64_t>(1, (uint64_t)c->num_sms * std::max(vper, 1)), 256, vsm,
                               s>>>(va, ent, slow, scal + Scal::NSLOW), FAST_LAUNCHED(c);
            stage_mark(c, 15, s);
            if ((st = read_scal(c, s, "row votes"))) return st;
            if (!single) {  // the single pass's writes were timed with it
                c->stats.ms_k_pairs += stage_ms(c, 10, 12);
                c->stats.ms_k_medium += stage_ms(c, 12, 11);
            }
            c->stats.ms_k_vote += stage_ms(c, 13, 14);
            c->stats.ms_k_vote_block += stage_ms(c, 14, 15);
            const uint64_t nlong = c->h_scal[Scal::NLONG];
            if (nlong > N) return set_error(c, FAST_EINTERNAL, "long-row list overflow");
            c->stats.n_long_rows += nlong;
            if (nlong) {
                std::vector<uint2> hl(nlong);
                cudaMemcpyAsync(hl.data(), long_rows, nlong * sizeof(uint2), cudaMemcpyDeviceToHost, s);
                if ((st = sync_check(c, s, "long rows"))) return st;
                // rows too long for a shared-memory hash use one in global
                // memory; their scratch is handed out chunk by chunk of rows,
                // at most kHugeWords words per launch (or one row's need)
                // (halved while the device cannot hold that much)
                constexpr uint64_t kHugeWords = 1ull << 29;
                std::vector<uint64_t> gofs(nlong), chunk;
                for (uint64_t r = 0; r < nlong; r++) c->stats.max_row = std::max<uint64_t>(c->stats.max_row, hl[r].y);
                for (uint64_t lim = kHugeWords, first = 1;; lim /= 2, first = 0) {
                    chunk.assign(1, 0);
                    uint64_t gtot = 0, gmax = 0, rmax = 0;
                    for (uint64_t r = 0; r < nlong; r++) {
                        uint64_t slots = 32;
                        while (slots < 2ull * hl[r].y) slots <<= 1;
                        const uint64_t need = slots > kRowBlockSlots ? 2 * slots : 0;
                        if (need && gtot + need > lim && gtot) {  // the next chunk starts here
                            chunk.push_back(r);
                            gtot = 0;
                        }
                        gofs[r] = gtot;
                        gtot += need;
                        gmax = std::max(gmax, gtot);
                        rmax = std::max(rmax, need);
                        if (first) c->stats.n_huge_rows += need != 0;
                    }
                    chunk.push_back(nlong);
                    if (gmax <= gscr_cap) break;  // one scratch for every partition, grown only when needed
                    dfree(c, gscr, gscr_cap * 4, s);
                    gscr = nullptr;
                    gscr_cap = 0;
                    if (!(st = dalloc_t(c, &gscr, gmax, s))) {
                        gscr_cap = gmax;
                        break;
                    }
                    if ((st != FAST_ENOMEM && st != FAST_EBUDGET) || lim <= rmax) return st;
                    st = FAST_OK;
                    c->err.clear();
                }
                cudaMemcpyAsync(d_gofs, gofs.data(), nlong * 8, cudaMemcpyHostToDevice, s);
                for (size_t k = 0; k + 1 < chunk.size(); k++) {
                    const uint64_t r0 = chunk[k], nr = chunk[k + 1] - r0;
                    stage_mark(c, 20, s);
                    k_long_vote<PT><<<(unsigned)std::min<uint64_t>(nr, c->num_sms * 2), 512, rsm, s>>>(
                        va, ent, long_rows + r0, nr, gscr, d_gofs + r0), FAST_LAUNCHED(c);
                    stage_mark(c, 21, s);
                    if ((st = read_scal(c, s, "long rows"))) return st;
                    c->stats.ms_k_vote_block += stage_ms(c, 20, 21);
                }
            }
        }
        const uint64_t used = c->h_scal[Scal::CUR_SPARSE];
        if (used <= sp_cap) {
            sp.keep = true;
            *sp_j_out = sp.j;
            *sp_v_out = sp.v;
            *sp_n_out = sp.n;
            return FAST_OK;
        }
        if (attempt == 1) break;
        sp_cap = used;  // exact size for the second pass
    }
    return set_error(c, FAST_EINTERNAL, "sparse list overflow");
}

// Row-partitioned search: dense groups, per-row sparse votes, row-ordered
// output with no global sort.
static fast_status search_rows(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, fast_result **out,
                               cudaStream_t s) {
    const fast_params &p = c->p;
    const uint64_t N = tb->N;
    const uint32_t nb = p.b;
    fast_status st = FAST_OK;
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
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
    auto fail = [&](fast_status r) {
        release();
        return r;
    };
    c->stats.n_fingerprints = N;
    c->stats.n_dropped = tb->n_dropped;
    c->stats.n_long_rows = c->stats.n_huge_rows = c->stats.max_row = 0;
    c->stats.query_parts = 1;
    c->stats.dense_fallback = 0;
    c->stats.group_shift = c->stats.region_slots = 0;
    uint32_t large_min = large_min_for(c, N);
    const unsigned blocksN = std::max(1u, std::min<unsigned>(ceil_div(N, 256), c->num_sms * 8));
    // A batch with the automatic threshold: one threshold per station, from
    // the station's own size and largest bucket (the batch's total would
    // turn a station's dense buckets into medium ones).  large_min is then
    // the largest of them.
    const uint32_t nst = tb->nst;
    const bool per_st = nst > 1 && !c->large_min;
    std::vector<uint32_t> lm_h;
    uint32_t *d_lm = nullptr;
    unsigned long long *d_lmax = nullptr;
    auto station_host = [&](uint64_t pos) {
        return (uint32_t)(std::upper_bound(tb->soff.begin(), tb->soff.end(), pos) - tb->soff.begin() - 1);
    };
    auto upload_lm = [&]() {
        cudaMemcpyAsync(d_lm, lm_h.data(), nst * 4, cudaMemcpyHostToDevice, s);
        large_min = *std::max_element(lm_h.begin(), lm_h.end());
    };

    // ---- big buckets
    stage_mark(c, 3, s);
    cudaMemsetAsync(scal, 0, sizeof(uint64_t) * kScal, s);
    // big buckets: found with the filter when the tables were built
    const uint64_t big_cap = tb->big_cap;
    uint4 *big = tb->d_big, *large = nullptr, *medium = nullptr;
    EnumArgs ea{tb->d_skey, tb->d_sid, tb->d_drop, nullptr, nullptr, N, p.excl, 0, (uint32_t)N, 1, {tb->d_soff, tb->nst}};
    cudaMemcpyAsync(scal + Scal::NBIG, tb->d_bigcnt, 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(scal + Scal::SMALLPAIRS, tb->d_bigcnt + 1, 8, cudaMemcpyDeviceToDevice, s);
    if ((st = read_scal(c, s, "bucket scan"))) return fail(st);
    const uint64_t nbig = c->h_scal[Scal::NBIG];
    if ((st = alloc(&large, nbig)) || (st = alloc(&medium, nbig))) return fail(st);
    const unsigned cg = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(nbig, c->num_sms * 8));
    if (per_st) {
        lm_h.resize(nst);
        for (uint32_t x = 0; x < nst; x++) lm_h[x] = large_min_for(c, tb->soff[x + 1] - tb->soff[x]);
        if ((st = alloc(&d_lm, nst)) || (st = alloc(&d_lmax, nst))) return fail(st);
        upload_lm();
        cudaMemsetAsync(d_lmax, 0, nst * 8, s);
    }
    k_big_classify<<<cg, 256, 0, s>>>(ea, big, scal + Scal::NBIG, big_cap, large_min, large, scal + Scal::NLARGE,
                                      medium, scal + Scal::NMEDIUM, scal + Scal::PART0, scal + Scal::LMAX, d_lm,
                                      d_lmax),
        FAST_LAUNCHED(c);
    if ((st = read_scal(c, s, "bucket classify"))) return fail(st);
    auto reclassify = [&]() {
        cudaMemsetAsync(scal + Scal::NLARGE, 0, 8, s);
        cudaMemsetAsync(scal + Scal::NMEDIUM, 0, 8, s);
        cudaMemsetAsync(scal + Scal::PART0, 0, 8 * (kScal - Scal::PART0), s);
        k_big_classify<<<cg, 256, 0, s>>>(ea, big, scal + Scal::NBIG, big_cap, large_min, large,
                                          scal + Scal::NLARGE, medium, scal + Scal::NMEDIUM, scal + Scal::PART0,
                                          nullptr, d_lm),
            FAST_LAUNCHED(c);
        return read_scal(c, s, "bucket classify");
    };
    // Automatic threshold, second bound: a dense group pays when its buckets
    // are a sizeable part of the largest one.  Buckets far below it only chain
    // windows that rarely reach v votes into one group whose pairs are all
    // compared (measured: a 31,104,000-window station 4.3 s -> 1.6 s, the
    // 7,776,000-window one 75.1 -> 73.8 ms, with identical lists).
    if (per_st) {
        std::vector<unsigned long long> lmx(nst);
        cudaMemcpyAsync(lmx.data(), d_lmax, nst * 8, cudaMemcpyDeviceToHost, s);
        if ((st = sync_check(c, s, "largest buckets"))) return fail(st);
        bool raised = false;
        for (uint32_t x = 0; x < nst; x++)
            if (lmx[x] / kLargeRel > lm_h[x]) {
                lm_h[x] = (uint32_t)(lmx[x] / kLargeRel);
                raised = true;
            }
        if (raised) {
            upload_lm();
            if ((st = reclassify())) return fail(st);
        }
    } else if (!c->large_min && c->h_scal[Scal::LMAX] / kLargeRel > large_min) {
        large_min = (uint32_t)(c->h_scal[Scal::LMAX] / kLargeRel);
        if ((st = reclassify())) return fail(st);
    }
    uint64_t nlarge = c->h_scal[Scal::NLARGE], nmedium = c->h_scal[Scal::NMEDIUM];

    // ---- dense groups: labels, members, keys, tile schedule, per-row counts
    uint32_t *label = nullptr, *GT = nullptr, *ids = nullptr, *dense_cnt = nullptr;
    uint64_t nm = 0, dense_pairs = 0, ngroups = 0, max_group = 0;
    std::vector<DenseTile> tiles;
    std::vector<DenseStrip> strips;
    uchar4 *tvotes = nullptr;  // votes of every dense tile, 64 x 64 bytes each
    DenseTile *d_tiles = nullptr;
    DenseStrip *d_strips = nullptr;
    const size_t dsm = (size_t)2 * nb * kDT * 4;
    if ((st = alloc(&label, N)) || (st = alloc(&dense_cnt, N))) return fail(st);
    cudaMemsetAsync(dense_cnt, 0, N * 4, s);
    std::vector<uint64_t> hm;
    uint64_t *sorted = nullptr;  // members as (group << 32 | id), sorted
    std::vector<std::pair<void *, size_t>> round_bufs;  // the last grouping round's member buffers
    struct RoundGuard {
        fast_ctx *c;
        cudaStream_t s;
        std::vector<std::pair<void *, size_t>> &v;
        ~RoundGuard() {
            for (auto &b : v) dfree(c, b.first, b.second, s);
        }
    } round_guard{c, s, round_bufs};
    // Groups are the connected components of the large buckets.  With the
    // automatic threshold a group must stay dense: comparing all its member
    // pairs may not cost more than the large buckets' own pairs (which the
    // sparse path would count); a group chained from many mid-size buckets
    // fails that, and the threshold doubles (measured on a 40,000,000-window
    // station of the 5-year shape: one 465,786-member group, 1.1e11 pair
    // comparisons, 2.55 s; after the check a 12,641-member group, 1.35 s;
    // identical lists).
    for (int round = 0;; round++) {
        cudaMemsetAsync(label, 0xFF, N * 4, s);
        nm = 0;
        hm.clear();
        if (!nlarge) break;
        const unsigned lg = (unsigned)std::min<uint64_t>(nlarge, c->num_sms * 8);
        k_label_init<<<lg, 256, 0, s>>>(large, nlarge, tb->d_sid, tb->d_drop, N, label), FAST_LAUNCHED(c);
        int it = 0;
        for (; it < 256; it++) {
            cudaMemsetAsync(scal + Scal::CHANGED, 0, 8, s);
            k_label_prop<<<lg, 256, 0, s>>>(large, nlarge, tb->d_sid, tb->d_drop, N, label,
                                            reinterpret_cast<uint32_t *>(scal + Scal::CHANGED)), FAST_LAUNCHED(c);
            if ((st = read_scal(c, s, "group labels"))) return fail(st);
            if (!c->h_scal[Scal::CHANGED]) break;
        }
        if (it == 256) return fail(set_error(c, FAST_EINTERNAL, "group labels did not converge"));
        cudaMemsetAsync(scal + Scal::NMEMB, 0, 8, s);
        for (auto &b : round_bufs) dfree(c, b.first, b.second, s);  // the previous round's members
        round_bufs.clear();
        unsigned long long *memb = nullptr, *memb2 = nullptr;
        if ((st = dalloc_t(c, &memb, N, s))) return fail(st);
        round_bufs.push_back({(void *)memb, N * 8});
        k_collect_members<<<blocksN, 256, 0, s>>>(label, N, memb, scal + Scal::NMEMB), FAST_LAUNCHED(c);
        if ((st = read_scal(c, s, "group members"))) return fail(st);
        nm = c->h_scal[Scal::NMEMB];
        if ((st = dalloc_t(c, &memb2, nm ? nm : 1, s))) return fail(st);
        round_bufs.push_back({(void *)memb2, (nm ? nm : 1) * 8});
        if ((st = sort_u64(c, nm, reinterpret_cast<uint64_t *>(memb), reinterpret_cast<uint64_t *>(memb2), 0,
                           32 + bits_for(N), &sorted, s)))
            return fail(st);
        hm.resize(nm);
        std::vector<uint4> hl(nlarge);
        cudaMemcpyAsync(hm.data(), sorted, nm * 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hl.data(), large, nlarge * sizeof(uint4), cudaMemcpyDeviceToHost, s);
        if ((st = sync_check(c, s, "group members copy"))) return fail(st);
        if (c->large_min || round >= 8) break;
        // member pairs of the groups, pairs of the large buckets (per station
        // in a batch: groups never cross stations)
        std::vector<uint64_t> gp(per_st ? nst : 1, 0), lp(per_st ? nst : 1, 0);
        for (uint64_t g0 = 0, g1; g0 < nm; g0 = g1) {
            for (g1 = g0 + 1; g1 < nm && (hm[g1] >> 32) == (hm[g0] >> 32); g1++) {
            }
            gp[per_st ? station_host((uint32_t)hm[g0]) : 0] += (g1 - g0) * (g1 - g0 - 1) / 2;
        }
        for (const uint4 &e : hl) lp[per_st ? station_host(e.y) : 0] += (uint64_t)e.w * (e.w - 1) / 2;
        auto twice = [](uint32_t m) { return m < (1u << 30) ? 2 * m : m + 1; };
        bool raised = false;
        for (size_t x = 0; x < gp.size(); x++)
            if (gp[x] > lp[x]) {  // and classify again
                if (per_st) lm_h[x] = twice(lm_h[x]);
                else large_min = twice(large_min);
                raised = true;
            }
        if (!raised) break;
        if (per_st) upload_lm();
        if ((st = reclassify())) return fail(st);
        nlarge = c->h_scal[Scal::NLARGE];
        nmedium = c->h_scal[Scal::NMEDIUM];
    }
    c->stats.large_min = large_min;
    for (auto &b : round_bufs) owned.push_back(b);  // `sorted` lives in them: freed with the search's buffers
    round_bufs.clear();
    stage_mark(c, 4, s);
    if (nlarge) {
        if ((st = alloc(&GT, (size_t)nm * nb)) || (st = alloc(&ids, nm))) return fail(st);
        k_gather_keys<<<std::max(1u, std::min<unsigned>(ceil_div(nm, 128), c->num_sms * 8)), 128, 0, s>>>(
            reinterpret_cast<unsigned long long *>(sorted), nm, d_sig, N, nb, GT, ids), FAST_LAUNCHED(c);
        std::vector<DenseGroup> hgrp;
        std::vector<uint32_t> htg, hmg(nm);  // group of each tile, of each member
        uint64_t g0 = 0;
        while (g0 < nm) {
            uint64_t g1 = g0 + 1;
            while (g1 < nm && (hm[g1] >> 32) == (hm[g0] >> 32)) g1++;
            const uint32_t n = (uint32_t)(g1 - g0);
            ngroups++;
            dense_pairs += (uint64_t)n * (n - 1) / 2;
            max_group = std::max<uint64_t>(max_group, n);
            const uint32_t gt0 = (uint32_t)tiles.size();  // the group's first tile
            const uint32_t nt = (n + kDT - 1) / kDT;
            hgrp.push_back({(uint32_t)g0, n, gt0, nt});
            for (uint64_t k = g0; k < g1; k++) hmg[k] = (uint32_t)hgrp.size() - 1;
            for (uint32_t a = 0; a < nt; a++) {
                strips.push_back({(uint32_t)g0, n, a, gt0});
                for (uint32_t b = a; b < nt; b++) {
                    tiles.push_back({(uint32_t)g0, n, a, b});
                    htg.push_back((uint32_t)hgrp.size() - 1);
                }
            }
            g0 = g1;
        }
        // longest strips first: they bound the emit pass
        std::stable_sort(strips.begin(), strips.end(), [](const DenseStrip &x, const DenseStrip &y) {
            return (x.n + kDT - 1) / kDT - x.ta > (y.n + kDT - 1) / kDT - y.ta;
        });
        if ((st = alloc(&d_tiles, tiles.size())) || (st = alloc(&d_strips, strips.size()))) return fail(st);
        cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(DenseTile), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_strips, strips.data(), strips.size() * sizeof(DenseStrip), cudaMemcpyHostToDevice, s);
        if ((st = alloc(&tvotes, tiles.size() * (kDT * kDT / 4)))) return fail(st);
        cudaMemsetAsync(tvotes, 0, tiles.size() * (size_t)(kDT * kDT), s);
        // cluster masks and the small clusters' pair votes
        uint32_t *d_tg = nullptr, *d_mg = nullptr, *gcol = nullptr, *gover = nullptr, *MB = nullptr;
        DenseGroup *d_grp = nullptr;
        if ((st = alloc(&d_tg, tiles.size())) || (st = alloc(&d_mg, nm)) || (st = alloc(&d_grp, ngroups)) ||
            (st = alloc(&gcol, ngroups)) || (st = alloc(&gover, ngroups)))
            return fail(st);
        cudaMemcpyAsync(d_tg, htg.data(), htg.size() * 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_mg, hmg.data(), nm * 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_grp, hgrp.data(), ngroups * sizeof(DenseGroup), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(gcol, 0, ngroups * 4, s);
        const uint64_t ne = (uint64_t)nb * nm;
        // the cluster masks need 36 bytes of scratch per member and table;
        // without them (or past 2^24 members) every group is voted by direct
        // key comparison
        auto clusters = [&]() -> fast_status {
            unsigned long long *ca = nullptr, *cb = nullptr;
            uint32_t *flag = nullptr;
            uint64_t *cid = nullptr, *cst = nullptr;
            fast_status r;
            if ((r = alloc(&MB, (size_t)kClW * nm)) || (r = alloc(&ca, ne)) || (r = alloc(&cb, ne)) ||
                (r = alloc(&flag, ne)) || (r = alloc(&cid, ne + 1)) || (r = alloc(&cst, ne + 1)))
                return r;
            cudaMemsetAsync(gover, 0, ngroups * 4, s);
            cudaMemsetAsync(MB, 0, (size_t)kClW * nm * 4, s);
            const unsigned eg = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(ne, 256), c->num_sms * 8));
            k_clu_comp<<<eg, 256, 0, s>>>(GT, nm, nb, ca), FAST_LAUNCHED(c);
            uint64_t *srt = nullptr;  // by (table, key), members ascending within (stable)
            if ((r = sort_u64(c, ne, reinterpret_cast<uint64_t *>(ca), reinterpret_cast<uint64_t *>(cb), 24, 64,
                              &srt, s)))
                return r;
            const unsigned long long *sc = reinterpret_cast<const unsigned long long *>(srt);
            k_clu_mark<<<eg, 256, 0, s>>>(sc, ne, d_mg, flag), FAST_LAUNCHED(c);
            if ((r = scan_excl(c, flag, cid, ne, 1, cid + ne, s))) return r;
            k_clu_starts<<<eg, 256, 0, s>>>(flag, cid, ne, cid + ne, cst), FAST_LAUNCHED(c);
            uint32_t *hcnt = nullptr, *gthr = nullptr;
            unsigned long long *hpairs = nullptr;
            if ((r = alloc(&hcnt, ngroups * kClBins)) || (r = alloc(&hpairs, ngroups * kClBins)) ||
                (r = alloc(&gthr, ngroups)))
                return r;
            cudaMemsetAsync(hcnt, 0, ngroups * kClBins * 4, s);
            cudaMemsetAsync(hpairs, 0, ngroups * kClBins * 8, s);
            k_clu_hist<<<eg, 256, 0, s>>>(sc, cst, cid + ne, d_mg, hcnt, hpairs), FAST_LAUNCHED(c);
            k_clu_thr<<<(unsigned)std::max<uint64_t>(1, ceil_div(ngroups, 128)), 128, 0, s>>>(d_grp, ngroups, nb,
                                                                                            hcnt, hpairs, gthr, gover),
                FAST_LAUNCHED(c);
            k_clu_apply<<<c->num_sms * 8, 256, 0, s>>>(sc, cst, cid + ne, d_mg, d_grp, nm, gcol, gover, MB,
                                                       reinterpret_cast<uint32_t *>(tvotes), gthr), FAST_LAUNCHED(c);
            return FAST_OK;
        };
        // only a lack of memory (or a group too large for the masks) falls
        // back to direct comparison; any other failure is the call's error
        const fast_status cr = nm >= (1u << 24) || nb > 256 || !c->dense_masks ? FAST_EBUDGET : clusters();
        if (cr && cr != FAST_ENOMEM && cr != FAST_EBUDGET) return fail(cr);
        if (cr) {
            c->err.clear();
            MB = nullptr;
            cudaMemsetAsync(gover, 0x01, ngroups * 4, s);  // every group by direct comparison
            c->stats.dense_fallback = 1;
        }
        cudaFuncSetAttribute(k_dense_rowcount, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        const unsigned dg = (unsigned)std::min<uint64_t>(tiles.size(), (uint64_t)c->num_sms * 4);
        k_dense_rowcount<<<dg, 256, dsm, s>>>(d_tiles, tiles.size(), GT, ids, nm, nb, p.v, p.excl, dense_cnt,
                                              tvotes, d_tg, gover), FAST_LAUNCHED(c);
        if (MB)
            k_dense_rowcount_mask<<<(unsigned)std::min<uint64_t>(tiles.size(), (uint64_t)c->num_sms * 8), 256, 0, s>>>(
                d_tiles, tiles.size(), d_tg, gcol, gover, MB, nm, ids, p.v, p.excl, dense_cnt, tvotes),
                FAST_LAUNCHED(c);
    }
    stage_mark(c, 5, s);
    sig_release(c, s);  // the keys are not read past the dense groups: their memory goes to the pairs

    // ---- sparse pairs: group-partitioned emission, per-row votes
    ea.label = label;
    {  // flagged copy of the id lists (made by the counting pass): the pair passes look up drop / label only for flagged ids
        uint32_t *bits = nullptr, *fsid = nullptr;
        const uint64_t n = (uint64_t)nb * N;
        if ((st = alloc(&bits, (N + 31) / 32))) return fail(st);
        // the copy saves the pair passes' bitmap lookups (the bitmap, N/8
        // bytes, mostly stays in L2) but costs b * N * 4 bytes: it is made
        // only when that is a small part of the memory left (the pair buffer
        // needs the rest); without it the passes read the bitmap
        if (n * 64 <= room_bytes(c) && alloc(&fsid, n)) {
            fsid = nullptr;
            c->err.clear();
        }
        k_flag_bits<<<std::max(1u, std::min<unsigned>(ceil_div((N + 31) / 32, 256), c->num_sms * 8)), 256, 0, s>>>(
            tb->d_drop, label, N, bits), FAST_LAUNCHED(c);
        ea.fbits = bits;      // the counting pass fills fsid,
        ea.fsid_out = fsid;   // the writing pass reads it
        ea.fsid = fsid;
    }
    uint32_t *sp_cnt = nullptr, *sp_j = nullptr;
    uint64_t *sp_start = nullptr;
    uint8_t *sp_v = nullptr;
    uint2 *long_rows = nullptr;
    if ((st = alloc(&sp_cnt, N)) || (st = alloc(&sp_start, N)) || (st = alloc(&long_rows, N))) return fail(st);
    uint64_t S = 0;
    {
        const uint64_t S_ub = c->h_scal[Scal::SMALLPAIRS] + c->h_scal[Scal::PART0];
        const double avg = (double)S_ub / (double)N;
        const uint32_t nbits = bits_for(N);
        uint32_t gshift = 0;
        const uint32_t target = c->group_pairs ? c->group_pairs : kVTargetDefault;
        while (gshift < 12 && (double)(2ull << gshift) * avg <= target) gshift++;
        // a batch's rows are not equally dense: background pairs per row grow
        // with the station's length, so station x expects N_x N / sum N_y^2
        // times the mean
        double dens = 1.0, sq = 0.0;
        for (uint32_t x = 0; x < nst; x++) sq += std::pow((double)(tb->soff[x + 1] - tb->soff[x]), 2);
        if (nst > 1 && sq > 0)
            for (uint32_t x = 0; x < nst; x++)
                dens = std::max(dens, (double)(tb->soff[x + 1] - tb->soff[x]) * (double)N / sq);
        // 32-bit entries while entry + 1 cannot wrap to the empty key
        uint64_t sp_n = 0;
        const fast_status r = gshift + nbits < 32
                                  ? sparse_groups<uint32_t>(c, ea, medium, nmedium, large_min, dens, gshift, nbits,
                                                            sp_cnt, sp_start, &sp_j, &sp_v, &sp_n, long_rows, S,
                                                            alloc, s, S_ub)
                                  : sparse_groups<unsigned long long>(c, ea, medium, nmedium, large_min, dens, gshift,
                                                                      nbits, sp_cnt, sp_start, &sp_j, &sp_v, &sp_n,
                                                                      long_rows, S, alloc, s, S_ub);
        if (r) return fail(r);
        owned.push_back({(void *)sp_j, sp_n * 4});  // freed with the search's other buffers
        owned.push_back({(void *)sp_v, sp_n});
    }
    stage_mark(c, 6, s);

    // ---- row offsets and the canonical list
    uint32_t *row_tot = nullptr;
    uint64_t *row_off = nullptr;
    if ((st = alloc(&row_tot, N)) || (st = alloc(&row_off, N + 1))) return fail(st);
    k_add_u32<<<blocksN, 256, 0, s>>>(dense_cnt, sp_cnt, row_tot, N), FAST_LAUNCHED(c);
    if ((st = scan_excl(c, row_tot, row_off, N, 1, row_off + N, s))) return fail(st);
    uint64_t M = 0;
    cudaMemcpyAsync(&M, row_off + N, 8, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "row offsets"))) return fail(st);
    stage_mark(c, 7, s);
    fast_result *res = new fast_result();
    res->ctx = c;
    res->stream = s;
    res->M = M;
    if ((st = dalloc_t(c, &res->d_i, M ? M : 1, s)) || (st = dalloc_t(c, &res->d_j, M ? M : 1, s)) ||
        (st = dalloc_t(c, &res->d_votes, M ? M : 1, s))) {
        fast_result_free(res);
        return fail(st);
    }
    if (!strips.empty())
        k_dense_rows<<<(unsigned)std::min<uint64_t>(strips.size(), (uint64_t)c->num_sms * 8), 256, 0, s>>>(
            d_strips, strips.size(), tvotes, ids, p.v, p.excl, row_off, res->d_i, res->d_j, res->d_votes),
            FAST_LAUNCHED(c);
    uint32_t *merge_rows = reinterpret_cast<uint32_t *>(long_rows);  // reuse: the long-row list is consumed
    uint64_t *mofs = nullptr;
    if ((st = alloc(&mofs, N))) {
        fast_result_free(res);
        return fail(st);
    }
    cudaMemsetAsync(scal + Scal::NMERGE, 0, 16, s);
    k_sparse_place<<<blocksN, 256, 0, s>>>(N, sp_cnt, sp_start, sp_j, sp_v, dense_cnt, row_off, res->d_i, res->d_j,
                                           res->d_votes, merge_rows, mofs, scal + Scal::NMERGE,
                                           scal + Scal::NMERGE_TOT), FAST_LAUNCHED(c);
    if ((st = read_scal(c, s, "sparse placement"))) {
        fast_result_free(res);
        return fail(st);
    }
    const uint64_t nmerge = c->h_scal[Scal::NMERGE], mtot = c->h_scal[Scal::NMERGE_TOT];
    if (nmerge) {
        uint32_t *tj = nullptr;
        uint8_t *tv = nullptr;
        if ((st = alloc(&tj, mtot)) || (st = alloc(&tv, mtot))) {
            fast_result_free(res);
            return fail(st);
        }
        k_row_merge<<<(unsigned)std::min<uint64_t>(nmerge, c->num_sms * 8), 256, 0, s>>>(
            merge_rows, nmerge, dense_cnt, sp_cnt, row_off, res->d_j, res->d_votes, tj, tv, mofs), FAST_LAUNCHED(c);
    }
    release();
    stage_mark(c, 8, s);
    if ((st = sync_check(c, s, "search output"))) {
        fast_result_free(res);
        return st;
    }
    c->stats.n_emissions = S;
    c->stats.n_dense_pairs = dense_pairs;
    c->stats.n_groups = ngroups;
    c->stats.max_group = max_group;
    c->stats.n_detections = M;
    c->stats.map_slots = 0;
    *out = res;
    return FAST_OK;
}

// Bit m of large bucket x's bitmap: member m of the bucket's group (members
// of a group sorted by id) belongs to the bucket.
__global__ void k_bucket_bitmaps(const uint4 *__restrict__ large, uint64_t nlarge, const uint32_t *__restrict__ sid,
                                 const uint8_t *__restrict__ drop, uint64_t N, const uint32_t *__restrict__ gstart,
                                 const uint32_t *__restrict__ ids, uint32_t *__restrict__ bm,
                                 const uint64_t *__restrict__ bm_off) {
    for (uint64_t x = blockIdx.x; x < nlarge; x += gridDim.x) {
        const uint4 e = large[x];
        const uint32_t *s = sid + (uint64_t)e.x * N;
        const uint32_t *gi = ids + gstart[e.w];
        const uint32_t gn = gstart[e.w + 1] - gstart[e.w];
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) {
            const uint32_t id = s[q];
            if (drop[id]) continue;
            uint32_t lo = 0, hi = gn;  // position of id among the group's sorted members
            while (lo < hi) {
                const uint32_t m = (lo + hi) / 2;
                if (gi[m] < id) lo = m + 1;
                else hi = m;
            }
            if (lo < gn && gi[lo] == id) atomicOr(bm + bm_off[x] + lo / 32, 1u << (lo % 32));
        }
    }
}

void history_groups_free(HistGroups *g) {
    cudaFree(g->label);
    cudaFree(g->ids);
    cudaFree(g->GT);
    cudaFree(g->gstart);
    cudaFree(g->large);
    cudaFree(g->tstart);
    cudaFree(g->bm);
    cudaFree(g->bm_off);
    *g = HistGroups{};
}

fast_status history_groups(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, HistGroups *g, cudaStream_t s) {
    const fast_params &p = c->p;
    const uint64_t N = tb->N;
    const uint32_t nb = p.b;
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
    fast_status st;
    *g = HistGroups{};
    const uint32_t large_min = large_min_for(c, N);
    g->large_min = large_min;
    auto dev = [&](auto **ptr, size_t count) -> fast_status {
        cudaError_t e = cudaMalloc(ptr, std::max<size_t>(count, 1) * sizeof(**ptr));
        return e ? cuda_fail(c, e, "history groups") : FAST_OK;
    };
    if ((st = dev(&g->label, N)) || (st = dev(&g->tstart, nb + 1))) return st;
    cudaMemsetAsync(g->label, 0xFF, N * 4, s);
    if (N == 0) {
        cudaMemsetAsync(g->tstart, 0, (nb + 1) * 4, s);
        return sync_check(c, s, "history groups");
    }
    const uint64_t big_cap = (uint64_t)nb * (N / (kSmall + 1) + 1);
    uint4 *big = nullptr, *large = nullptr, *medium = nullptr;
    if ((st = dalloc_t(c, &big, big_cap, s))) return st;
    cudaMemsetAsync(scal, 0, sizeof(uint64_t) * kScal, s);
    EnumArgs ea{tb->d_skey, tb->d_sid, tb->d_drop, nullptr, nullptr, N, p.excl, 0, (uint32_t)N, 1, {tb->d_soff, tb->nst}};
    const uint32_t ftpw = tiles_per_warp(c, N, nb);
    const dim3 eg((unsigned)std::max<uint64_t>(1, (((N + 31) / 32 + ftpw - 1) / ftpw + 7) / 8), nb);
    k_find_big<<<eg, 256, 0, s>>>(ea, ftpw, big, scal + Scal::NBIG, big_cap, scal + Scal::SMALLPAIRS, c->d_err),
        FAST_LAUNCHED(c);
    if ((st = read_scal(c, s, "history buckets"))) {
        dfree(c, big, big_cap * 16, s);
        return st;
    }
    const uint64_t nbig = c->h_scal[Scal::NBIG];
    if ((st = dalloc_t(c, &large, nbig ? nbig : 1, s)) || (st = dalloc_t(c, &medium, nbig ? nbig : 1, s))) {
        dfree(c, big, big_cap * 16, s);
        return st;
    }
    k_big_classify<<<std::max<uint64_t>(1, std::min<uint64_t>(nbig, c->num_sms * 8)), 256, 0, s>>>(
        ea, big, scal + Scal::NBIG, big_cap, large_min, large, scal + Scal::NLARGE, medium, scal + Scal::NMEDIUM,
        scal + Scal::PART0), FAST_LAUNCHED(c);
    st = read_scal(c, s, "history classify");
    const uint64_t nlarge = c->h_scal[Scal::NLARGE];
    std::vector<uint4> hl(nlarge);
    if (!st && nlarge) {
        const unsigned lg = (unsigned)std::min<uint64_t>(nlarge, c->num_sms * 8);
        k_label_init<<<lg, 256, 0, s>>>(large, nlarge, tb->d_sid, tb->d_drop, N, g->label), FAST_LAUNCHED(c);
        int it = 0;
        for (; it < 256 && !st; it++) {
            cudaMemsetAsync(scal + Scal::CHANGED, 0, 8, s);
            k_label_prop<<<lg, 256, 0, s>>>(large, nlarge, tb->d_sid, tb->d_drop, N, g->label,
                                            reinterpret_cast<uint32_t *>(scal + Scal::CHANGED)), FAST_LAUNCHED(c);
            st = read_scal(c, s, "history labels");
            if (!st && !c->h_scal[Scal::CHANGED]) break;
        }
        if (!st && it == 256) st = set_error(c, FAST_EINTERNAL, "group labels did not converge");
        cudaMemcpyAsync(hl.data(), large, nlarge * sizeof(uint4), cudaMemcpyDeviceToHost, s);
    }
    dfree(c, big, big_cap * 16, s);
    dfree(c, large, (nbig ? nbig : 1) * 16, s);
    dfree(c, medium, (nbig ? nbig : 1) * 16, s);
    if (st) return st;
    // members sorted by (label, id)
    unsigned long long *memb = nullptr, *memb2 = nullptr;
    if ((st = dalloc_t(c, &memb, N, s))) return st;
    cudaMemsetAsync(scal + Scal::NMEMB, 0, 8, s);
    k_collect_members<<<std::max(1u, std::min<unsigned>(ceil_div(N, 256), c->num_sms * 8)), 256, 0, s>>>(
        g->label, N, memb, scal + Scal::NMEMB), FAST_LAUNCHED(c);
    if ((st = read_scal(c, s, "history members"))) {
        dfree(c, memb, N * 8, s);
        return st;
    }
    const uint64_t nm = c->h_scal[Scal::NMEMB];
    g->nm = nm;
    std::vector<uint64_t> hm(nm);
    if (nm) {
        if ((st = dalloc_t(c, &memb2, nm, s))) {
            dfree(c, memb, N * 8, s);
            return st;
        }
        uint64_t *sorted = nullptr;
        st = sort_u64(c, nm, reinterpret_cast<uint64_t *>(memb), reinterpret_cast<uint64_t *>(memb2), 0,
                      32 + bits_for(N), &sorted, s);
        if (!st) st = dev(&g->GT, (size_t)nm * nb);
        if (!st) st = dev(&g->ids, nm);
        if (!st) {
            cudaMemcpyAsync(hm.data(), sorted, nm * 8, cudaMemcpyDeviceToHost, s);
            k_gather_keys<<<std::max(1u, std::min<unsigned>(ceil_div(nm, 128), c->num_sms * 8)), 128, 0, s>>>(
                reinterpret_cast<unsigned long long *>(sorted), nm, d_sig, N, nb, g->GT, g->ids), FAST_LAUNCHED(c);
            st = sync_check(c, s, "history member keys");
        }
        dfree(c, memb2, nm * 8, s);
    }
    dfree(c, memb, N * 8, s);
    if (st) return st;
    // group table and the large buckets of every table with their group index
    std::vector<uint32_t> gstart, glabel;
    for (uint64_t a = 0; a < nm; a++)
        if (a == 0 || (hm[a] >> 32) != (hm[a - 1] >> 32)) {
            gstart.push_back((uint32_t)a);
            glabel.push_back((uint32_t)(hm[a] >> 32));
        }
    g->ng = gstart.size();
    gstart.push_back((uint32_t)nm);
    std::vector<uint32_t> hlabel(N);
    if (nlarge) cudaMemcpy(hlabel.data(), g->label, N * 4, cudaMemcpyDeviceToHost);
    std::vector<uint32_t> hsid;
    std::vector<uint4> lg;
    for (const uint4 &e : hl) {
        // the group of a large bucket: label of any live member (all share it)
        uint32_t lab = kNone;
        std::vector<uint32_t> ids_probe(std::min<uint32_t>(e.z - e.y, 64));
        cudaMemcpy(ids_probe.data(), tb->d_sid + (uint64_t)e.x * N + e.y, ids_probe.size() * 4, cudaMemcpyDeviceToHost);
        for (uint32_t id : ids_probe)
            if (hlabel[id] != kNone) {
                lab = hlabel[id];
                break;
            }
        if (lab == kNone) continue;
        const uint32_t gi = (uint32_t)(std::lower_bound(glabel.begin(), glabel.end(), lab) - glabel.begin());
        lg.push_back(make_uint4(e.x, e.y, e.z, gi));
    }
    std::sort(lg.begin(), lg.end(), [](const uint4 &a, const uint4 &b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
    // the resident per-window array holds the group index (not the label)
    if (nlarge) {
        for (uint64_t x = 0; x < N; x++)
            if (hlabel[x] != kNone)
                hlabel[x] = (uint32_t)(std::lower_bound(glabel.begin(), glabel.end(), hlabel[x]) - glabel.begin());
        cudaMemcpy(g->label, hlabel.data(), N * 4, cudaMemcpyHostToDevice);
    }
    std::vector<uint32_t> ts(nb + 1, 0);
    for (const uint4 &e : lg) ts[e.x + 1]++;
    for (uint32_t t = 0; t < nb; t++) ts[t + 1] += ts[t];
    g->nlarge = lg.size();
    std::vector<uint64_t> boff(lg.size() + 1, 0);
    for (size_t x = 0; x < lg.size(); x++) {
        const uint32_t gs = gstart[lg[x].w + 1] - gstart[lg[x].w];
        boff[x + 1] = boff[x] + (gs + 31) / 32;
    }
    if ((st = dev(&g->gstart, gstart.size())) || (st = dev(&g->large, lg.size())) ||
        (st = dev(&g->bm_off, lg.size() + 1)) || (st = dev(&g->bm, boff.back())))
        return st;
    cudaMemcpy(g->gstart, gstart.data(), gstart.size() * 4, cudaMemcpyHostToDevice);
    if (!lg.empty()) cudaMemcpy(g->large, lg.data(), lg.size() * sizeof(uint4), cudaMemcpyHostToDevice);
    cudaMemcpy(g->tstart, ts.data(), ts.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(g->bm_off, boff.data(), boff.size() * 8, cudaMemcpyHostToDevice);
    cudaMemsetAsync(g->bm, 0, std::max<uint64_t>(boff.back(), 1) * 4, s);
    if (!lg.empty())
        k_bucket_bitmaps<<<(unsigned)std::min<uint64_t>(lg.size(), c->num_sms * 8), 256, 0, s>>>(
            g->large, lg.size(), tb->d_sid, tb->d_drop, N, g->gstart, g->ids, g->bm, g->bm_off), FAST_LAUNCHED(c);
    return sync_check(c, s, "history groups");
}

fast_status search_run(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, fast_result **out,
                       cudaStream_t s) {
    if (tb->N == 0) {  // nothing to launch
        fast_result *res = new fast_result();
        res->ctx = c;
        res->stream = s;
        fast_status st;
        if ((st = dalloc_t(c, &res->d_i, 1, s)) || (st = dalloc_t(c, &res->d_j, 1, s)) ||
            (st = dalloc_t(c, &res->d_votes, 1, s))) {
            fast_result_free(res);
            return st;
        }
        c->stats = fast_stats{};
        *out = res;
        return FAST_OK;
    }
    c->stats.max_group = 0;
    c->stats.ms_k_pairs = c->stats.ms_k_medium = c->stats.ms_k_vote = c->stats.ms_k_vote_block = 0.f;
    c->stats.ms_k_count_small = c->stats.ms_k_count_medium = 0.f;
    return c->vote_map ? search_map(c, tb, d_sig, out, s) : search_rows(c, tb, d_sig, out, s);
}

}  // namespace fastgb
