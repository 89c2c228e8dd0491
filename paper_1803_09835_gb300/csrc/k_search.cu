// k_search.cu -- occurrence filter (§6.5), pair enumeration inside buckets and
// vote counting (§6.1 "Search", §6.3), threshold and canonical output (§7.2).
//
// votes(i, j) = number of tables in which i and j share a bucket; a pair is
// reported when neither is dropped, j - i > excl and votes >= v.
//
// GB300 design.  Every bucket pair is one "emission"; emissions from all b
// tables must be summed per pair.  Buckets come in two very different kinds:
//   * sparse: the background, sizes ~2..50, almost every pair seen once.
//     Their pairs are summed in a device open-addressing hash map of packed
//     (i, j) -> uint8 votes (one 64-bit slot: i:28 | j:28 | votes:8).
//   * dense: a repeating source (e.g. periodic noise) puts thousands of
//     near-copies in one bucket in most tables, so the same pairs recur in
//     every table -- ~10^10 emissions for ~10^8 distinct pairs.  Buckets with
//     at least `large_min` live members are merged into groups (connected
//     components of shared large buckets); for every pair inside a group the
//     votes are computed directly by comparing the two fingerprints' b keys,
//     tile by tile in shared memory, once per pair instead of once per table.
//     The sparse path skips pairs inside a group, so each pair is counted by
//     exactly one of the two paths, and both count exactly the definition.
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

// Heavy bucket starts: size >= smin, i.e. occ_den * size > occ_num * N.
__global__ void k_heavy_find(const uint32_t *__restrict__ skey, uint64_t N, uint64_t smin,
                             uint4 *__restrict__ list, unsigned long long *__restrict__ count, uint64_t cap,
                             uint32_t *err) {
    const uint32_t t = blockIdx.y;
    const uint32_t *k = skey + (uint64_t)t * N;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t key = k[p];
        if (p > 0 && k[p - 1] == key) continue;
        if (p + smin - 1 >= N || k[p + smin - 1] != key) continue;
        // gallop then bisect to the end of the run
        uint64_t lo = p + smin - 1, step = 1, hi;
        for (;;) {
            hi = lo + step;
            if (hi >= N || k[hi] != key) break;
            lo = hi;
            step <<= 1;
        }
        if (hi > N) hi = N;
        while (hi - lo > 1) {  // k[lo] == key, k[hi] != key or hi == N
            uint64_t mid = lo + (hi - lo) / 2;
            if (k[mid] == key) lo = mid;
            else hi = mid;
        }
        unsigned long long slot = atomicAdd(count, 1ull);
        if (slot < cap) list[slot] = make_uint4(t, (uint32_t)p, (uint32_t)hi, 0);
        else set_err(err, ERR_OVERFLOW);
    }
}

__global__ void k_heavy_mark(const uint4 *__restrict__ list, const unsigned long long *__restrict__ count,
                             uint64_t cap, const uint32_t *__restrict__ sid, uint64_t N, uint32_t *__restrict__ heavy) {
    const uint64_t n = min((uint64_t)*count, cap);
    for (uint64_t b = blockIdx.x; b < n; b += gridDim.x) {
        uint4 e = list[b];
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

// --------------------------------------------------- bucket enumeration

struct EnumArgs {
    const uint32_t *skey, *sid;
    const uint8_t *drop;
    const uint32_t *label;  // nullptr before grouping
    uint64_t N;
    uint32_t excl;
    uint32_t i_lo, i_hi;  // query partition [i_lo, i_hi)
    uint32_t nparts;      // counting: partition of i is i * nparts / N
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
        const uint32_t key = k[p];
        if (p > 0 && k[p - 1] == key) continue;
        uint64_t e = p + 1;
        while (e < N && e - p <= kSmall && k[e] == key) e++;
        if (e - p == 1) continue;
        if (e - p > kSmall) {
            if (MODE == 0) {
                uint64_t lo = e - 1, step = 1, hi;
                for (;;) {
                    hi = lo + step;
                    if (hi >= N || k[hi] != key) break;
                    lo = hi;
                    step <<= 1;
                }
                if (hi > N) hi = N;
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
// (each live member i pairs with the live members after it).
__global__ void __launch_bounds__(256) k_big_classify(EnumArgs a, const uint4 *__restrict__ big,
                                                      const unsigned long long *__restrict__ nbig, uint64_t big_cap,
                                                      uint32_t large_min, uint4 *__restrict__ large,
                                                      unsigned long long *__restrict__ nlarge, uint4 *__restrict__ medium,
                                                      unsigned long long *__restrict__ nmedium,
                                                      unsigned long long *__restrict__ part_cnt) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_live;
    __shared__ unsigned long long s_cnt[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) s_cnt[i] = 0;
    const uint64_t n = min((uint64_t)*nbig, big_cap);
    for (uint64_t bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const uint4 e = big[bi];
        const uint32_t *s = a.sid + (uint64_t)e.x * a.N;
        uint32_t live = 0;
        for (uint32_t q = e.y + threadIdx.x; q < e.z; q += blockDim.x) live += !a.drop[s[q]];
        for (int o = 16; o; o >>= 1) live += __shfl_down_sync(~0u, live, o);
        if (threadIdx.x == 0) s_live = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_live, live);
        __syncthreads();
        const uint32_t nl = s_live;
        if (threadIdx.x == 0 && nl >= 2) {
            if (nl >= large_min) large[atomicAdd(nlarge, 1ull)] = make_uint4(e.x, e.y, e.z, nl);
            else medium[atomicAdd(nmedium, 1ull)] = make_uint4(e.x, e.y, e.z, nl);
        }
        if (nl >= 2 && nl < large_min) {
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

uint32_t bits_for(uint64_t N) {
    uint32_t nb = 1;
    while (nb < 32 && (1ull << nb) < N) nb++;
    return nb;
}

struct Scal {  // device scalar slots (ctx->d_scal)
    enum { NBIG, NLARGE, NMEDIUM, NHEAVY, NDROP, NMEMB, CUR_DENSE, CUR_SPARSE, CHANGED, PART0 };
};

}  // namespace

// ------------------------------------------------------------ host side

fast_status filter_launch(fast_ctx *c, fast_tables *tb, cudaStream_t s) {
    const fast_params &p = c->p;
    const uint64_t N = tb->N;
    fast_status st;
    unsigned long long *scal = reinterpret_cast<unsigned long long *>(c->d_scal);
    cudaMemsetAsync(scal, 0, sizeof(uint64_t) * kScal, s);
    uint32_t *heavy = nullptr;
    if (p.occ_num > 0 && N > 0) {
        const uint64_t smin = (uint64_t)p.occ_num * N / p.occ_den + 1;  // heavy iff size >= smin
        const uint64_t cap = (uint64_t)p.b * (N / smin + 1);
        if (cap > (1ull << 26)) return set_error(c, FAST_EBUDGET, "occurrence threshold too small for this N");
        uint4 *list = nullptr;
        if ((st = dalloc_t(c, &heavy, N, s))) return st;
        if ((st = dalloc_t(c, &list, cap, s))) {
            dfree(c, heavy, N * 4, s);
            return st;
        }
        cudaMemsetAsync(heavy, 0, N * 4, s);
        dim3 g(std::max(1u, std::min<unsigned>(ceil_div(N, 256), 4096)), p.b);
        k_heavy_find<<<g, 256, 0, s>>>(tb->d_skey, N, smin, list, scal + Scal::NHEAVY, cap, c->d_err), FAST_LAUNCHED(c);
        k_heavy_mark<<<c->num_sms * 4, 256, 0, s>>>(list, scal + Scal::NHEAVY, cap, tb->d_sid, N, heavy), FAST_LAUNCHED(c);
        dfree(c, list, cap * sizeof(uint4), s);
    }
    k_drop<<<std::max(1u, std::min<unsigned>(ceil_div(N, 256), c->num_sms * 8)), 256, 0, s>>>(heavy, N, p.b, tb->d_drop,
                                                                                             scal + Scal::NDROP), FAST_LAUNCHED(c);
    if (heavy) dfree(c, heavy, N * 4, s);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(c, e, "filter");
    cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(uint64_t) * kScal, cudaMemcpyDeviceToHost, s);
    if ((st = sync_check(c, s, "occurrence filter"))) return st;
    tb->n_dropped = c->h_scal[Scal::NDROP];
    return FAST_OK;
}

static fast_status read_scal(fast_ctx *c, cudaStream_t s, const char *where) {
    cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(uint64_t) * kScal, cudaMemcpyDeviceToHost, s);
    return sync_check(c, s, where);
}

fast_status search_run(fast_ctx *c, const fast_tables *tb, const uint32_t *d_sig, fast_result **out,
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

    // large_min: above the largest bucket the random background makes.  The
    // most likely key of a table has probability ~(K/D)^r, so the background
    // tops out near N (K/D)^r members; take 8x that, at least 512.
    uint32_t large_min = c->large_min;
    if (!large_min) {
        double ptop = std::pow((double)p.K / p.D, (double)p.r);
        large_min = (uint32_t)std::max(512.0, std::min(1e9, 8.0 * N * ptop));
    }

    uint32_t nparts = p.query_part ? p.query_part : 1;
    nparts = std::min<uint32_t>(nparts, 64);

    // ---- pass 1: big buckets and small-pair counts
    stage_mark(c, 3, s);
    cudaMemsetAsync(scal, 0, sizeof(uint64_t) * kScal, s);
    const uint64_t big_cap = (uint64_t)nb * (N / (kSmall + 1) + 1);
    uint4 *big = nullptr, *large = nullptr, *medium = nullptr;
    if ((st = alloc(&big, big_cap))) return fail(st);
    EnumArgs ea{tb->d_skey, tb->d_sid, tb->d_drop, nullptr, N, p.excl, 0, (uint32_t)N, nparts};
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
    stage_mark(c, 5, s);

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
    stage_mark(c, 6, s);
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
    stage_mark(c, 7, s);

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

}  // namespace fastgb
