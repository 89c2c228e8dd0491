// k_sort.cu -- stable LSD radix sort used to build the hash tables
// (§6.1 "Hash table construction": each table maps a signature to the list
// of fingerprints sharing it) and to order the detection list.
//
// One launch sorts `nseg` equal-length segments (all b tables at once).
// Each 8-bit pass is reduce-then-scan, with no inter-CTA waits:
//   k_hist    per (segment, chunk) digit counts        -- reads keys
//   scan      per segment exclusive scan, digit-major (k_scan.cu)
//   k_scatter per chunk: stable rank of every key inside the chunk (peer
//             masks + per-warp counters in shared memory), staging in
//             shared memory in digit order, then coalesced runs written to
//             the digit's global position.
// Stability makes the ids of a bucket come out ascending, i.e. the canonical
// bucket listing (key ascending, id ascending).
#include <algorithm>
#include <mutex>

#include "fast_internal.cuh"

namespace fastgb {

namespace {

constexpr int kRadix = 256;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kSub = kThreads * kItems;  // 2048 keys per sub-tile
constexpr int kSubPerChunk = 3;
constexpr int kChunk = kSub * kSubPerChunk;  // 6144 keys per chunk (faster than 8192 on GB300: measured)

template <typename KT>
__device__ __forceinline__ uint32_t digit_of(KT k, uint32_t shift) {
    return (uint32_t)(k >> shift) & (kRadix - 1);
}

// Segment y of a sort: the y-th of nseg rows of `len` keys or, with several
// stations, row y / nst's keys of station y % nst: positions soff[x] ..
// soff[x + 1] of the row, whose generated ids start at soff[x].  Sorting
// every station's part of a table on its own leaves the table ordered by
// (station, key, id).
struct Seg {
    uint64_t base, n, id0;
};
__device__ __forceinline__ Seg seg_of(uint32_t y, uint64_t len, const Stations &S) {
    if (S.nst <= 1) return Seg{(uint64_t)y * len, len, 0};
    const uint32_t t = y / S.nst, x = y % S.nst;
    const uint64_t a = S.soff[x];
    return Seg{(uint64_t)t * len + a, S.soff[x + 1] - a, a};
}

template <typename KT>
__global__ void __launch_bounds__(kThreads) k_hist(const KT *__restrict__ keys, uint64_t len, uint32_t nchunks,
                                                   uint32_t shift, uint32_t *__restrict__ counts,
                                                   Stations S = Stations{nullptr, 1}) {
    __shared__ uint32_t h[kWarps][kRadix];
    const uint32_t seg = blockIdx.y, chunk = blockIdx.x;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const Seg g = seg_of(seg, len, S);
    const KT *k = keys + g.base;
    const uint64_t lo = (uint64_t)chunk * kChunk, hi = std::min<uint64_t>(lo + kChunk, g.n);
    const int warp = threadIdx.x >> 5;
    for (uint64_t e = lo + threadIdx.x; e < hi; e += kThreads) atomicAdd(&h[warp][digit_of(__ldcs(k + e), shift)], 1u);
    __syncthreads();
    uint32_t d = threadIdx.x, tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) tot += h[w][d];
    counts[((uint64_t)seg * kRadix + d) * nchunks + chunk] = tot;
}

// Exclusive scan over one segment's [digit][chunk] counts.
__global__ void __launch_bounds__(1024) k_scan(const uint32_t *__restrict__ counts, uint64_t *__restrict__ offsets,
                                               uint32_t nchunks) {
    __shared__ uint64_t wsum[32];
    const uint64_t n = (uint64_t)kRadix * nchunks;
    const uint32_t *c = counts + (uint64_t)blockIdx.x * n;
    uint64_t *o = offsets + (uint64_t)blockIdx.x * n;
    const uint64_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = std::min<uint64_t>(n, per * threadIdx.x), hi = std::min<uint64_t>(n, lo + per);
    uint64_t s = 0;
    for (uint64_t i = lo; i < hi; i++) s += c[i];
    // block exclusive scan of s
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(~0u, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(~0u, v, d);
            if (lane >= d) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    uint64_t run = x - s + (warp > 0 ? wsum[warp - 1] : 0);
    for (uint64_t i = lo; i < hi; i++) {
        o[i] = run;
        run += c[i];
    }
}

// Dynamic shared memory of k_scatter: the whole chunk staged in digit order.
template <typename KT, bool HAS_VAL>
constexpr size_t scatter_smem() {
    return (size_t)kChunk * (sizeof(KT) + (HAS_VAL ? 4 : 0));
}

// Staging of one chunk: (key, id) pairs interleaved for 32-bit keys (one
// 64-bit shared store per item), separate key and id arrays otherwise.
template <typename KT, bool HAS_VAL>
struct Staging {
    static constexpr bool kPair = HAS_VAL && sizeof(KT) == 4;
    unsigned long long *raw;
    __device__ __forceinline__ void put(uint32_t pos, KT k, uint32_t v) const {
        if constexpr (kPair) {
            reinterpret_cast<uint2 *>(raw)[pos] = make_uint2((uint32_t)k, v);
        } else {
            reinterpret_cast<KT *>(raw)[pos] = k;
            if (HAS_VAL) reinterpret_cast<uint32_t *>(reinterpret_cast<KT *>(raw) + kChunk)[pos] = v;
        }
    }
    __device__ __forceinline__ void get(uint32_t pos, KT &k, uint32_t &v) const {
        if constexpr (kPair) {
            const uint2 kv = reinterpret_cast<const uint2 *>(raw)[pos];
            k = (KT)kv.x;
            v = kv.y;
        } else {
            k = reinterpret_cast<const KT *>(raw)[pos];
            v = HAS_VAL ? reinterpret_cast<const uint32_t *>(reinterpret_cast<const KT *>(raw) + kChunk)[pos] : 0u;
        }
    }
};

// One chunk (6144 keys) per CTA.  The chunk's digit starts come from its
// k_hist counts; its three sub-tiles of 2048 are ranked one after another
// into a shared-memory copy of the chunk in digit order, which is then
// written out once: each digit's run (~24 keys) goes to run[d] onwards.
//
// Ranking of one item slot of a warp (32 keys, one per lane), stable by lane:
// every lane ORs its bit into the warp's mask word of its digit, reads the
// mask back (its peers: lanes with the same digit) together with the warp's
// running count of that digit, and the lowest peer clears the mask and
// advances the count.  Lanes before this one among its peers give its rank.
// Measured on GB300 this beats eight warp ballots per slot (the ballot pipe
// is the narrow one) and the match instruction (narrower still).
// The next sub-tile's loads are issued before the current one is ranked.
template <typename KT, bool HAS_VAL, bool IOTA>
__global__ void __launch_bounds__(kThreads, 3) k_scatter(const KT *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                      KT *__restrict__ kout, uint32_t *__restrict__ vout, uint64_t len,
                                                      uint32_t nchunks, uint32_t shift,
                                                      const uint32_t *__restrict__ counts,
                                                      const uint64_t *__restrict__ offsets,
                                                      Stations S = Stations{nullptr, 1}) {
    constexpr bool PF = sizeof(KT) == 4;  // register prefetch (64-bit keys would spill)
    extern __shared__ unsigned long long sc_raw[];
    const Staging<KT, HAS_VAL> stage{sc_raw};
    __shared__ uint64_t delta[kRadix];          // global position - chunk position, per digit
    __shared__ uint16_t wpos[kWarps][kRadix];   // per-warp counts, then per-warp chunk positions
    __shared__ uint32_t wmask[kWarps][kRadix];  // peer masks (zero between uses)
    __shared__ uint32_t cpos[kRadix], wscan[kWarps];

    const uint32_t seg = blockIdx.y, chunk = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1;
    const Seg g = seg_of(seg, len, S);
    const uint64_t cbase = (uint64_t)chunk * kChunk;
    if (cbase >= g.n) return;  // block-uniform: a station shorter than the longest
    const KT *ki = kin + g.base;
    const uint32_t *vi = HAS_VAL && !IOTA ? vin + g.base : nullptr;
    KT *ko = kout + g.base;
    uint32_t *vo = HAS_VAL ? vout + g.base : nullptr;
    const uint32_t cvalid = (uint32_t)std::min<uint64_t>(kChunk, g.n - cbase);
#pragma unroll
    for (int w = 0; w < kWarps; w++) wmask[w][threadIdx.x] = 0;
    {   // the chunk's digit starts: exclusive scan of its counts over the 256 digits
        const uint32_t d = threadIdx.x;
        const uint64_t run = offsets[((uint64_t)seg * kRadix + d) * nchunks + chunk];
        const uint32_t cnt = counts[((uint64_t)seg * kRadix + d) * nchunks + chunk];
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(~0u, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wscan[warp] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < warp; w++) add += wscan[w];
        const uint32_t cs = x - cnt + add;
        cpos[d] = cs;
        delta[d] = run - cs;
    }

    KT key[kItems], nkey[kItems];
    uint32_t val[kItems], nval[kItems];
    auto load = [&](uint64_t sb, KT *k, uint32_t *v) {
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint64_t e = sb + warp * (kItems * 32) + j * 32 + lane;
            const bool valid = e < g.n;
            // streaming loads (evict-first): the L2 keeps the write frontier of the digit runs
            k[j] = valid ? __ldcs(ki + e) : (KT)0;
            if (HAS_VAL) v[j] = valid ? (IOTA ? (uint32_t)(g.id0 + e) : __ldcs(vi + e)) : 0u;
        }
    };
#pragma unroll
    for (int sub = 0; sub < kSubPerChunk; sub++) {
        const uint64_t sbase = cbase + (uint64_t)sub * kSub;
        if (sbase >= g.n) break;  // block-uniform
        const uint32_t nvalid = (uint32_t)std::min<uint64_t>(kSub, g.n - sbase);
#pragma unroll
        for (int w = 0; w < kWarps; w++) wpos[w][threadIdx.x] = 0;
        if (!PF || sub == 0) load(sbase, key, val);
        if (PF && sub + 1 < kSubPerChunk) load(sbase + kSub, nkey, nval);
        __syncthreads();

        uint32_t rnk[kItems];
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t e = warp * (kItems * 32) + j * 32 + lane;
            const bool valid = e < nvalid;
            uint32_t dig = 0;
            if (valid) {
                dig = digit_of(key[j], shift);
                atomicOr(&wmask[warp][dig], 1u << lane);
            }
            __syncwarp();
            const uint32_t peers = valid ? wmask[warp][dig] : 0u;
            const uint32_t basec = valid ? wpos[warp][dig] : 0u;
            __syncwarp();
            const uint32_t before = peers & lt_mask;
            if (valid && before == 0) {
                wmask[warp][dig] = 0;
                wpos[warp][dig] = (uint16_t)(basec + __popc(peers));
            }
            __syncwarp();
            rnk[j] = basec + __popc(before);
        }
        __syncthreads();
        {   // per digit: chunk position of each warp's first key of that digit
            const uint32_t d = threadIdx.x;
            uint32_t r = cpos[d];
#pragma unroll
            for (int w = 0; w < kWarps; w++) {
                const uint32_t c = wpos[w][d];
                wpos[w][d] = (uint16_t)r;
                r += c;
            }
            cpos[d] = r;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t e = warp * (kItems * 32) + j * 32 + lane;
            if (e < nvalid) {
                const uint32_t dig = digit_of(key[j], shift);
                stage.put(wpos[warp][dig] + rnk[j], key[j], HAS_VAL ? val[j] : 0u);
            }
        }
        if (PF) {
#pragma unroll
            for (int j = 0; j < kItems; j++) {
                key[j] = nkey[j];
                val[j] = nval[j];
            }
        }
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < cvalid; i += kThreads) {
        KT k;
        uint32_t v;
        stage.get(i, k, v);
        const uint64_t o = delta[digit_of(k, shift)] + i;
        ko[o] = k;
        if (HAS_VAL) vo[o] = v;
    }
}

// Opt every k_scatter instantiation into its dynamic shared memory (once per
// process and device; the attribute outlives the call).
void scatter_attrs() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaFuncSetAttribute(k_scatter<uint32_t, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)scatter_smem<uint32_t, true>());
    cudaFuncSetAttribute(k_scatter<uint32_t, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)scatter_smem<uint32_t, true>());
    cudaFuncSetAttribute(k_scatter<uint64_t, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)scatter_smem<uint64_t, false>());
    cudaFuncSetAttribute(k_scatter<uint64_t, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)scatter_smem<uint64_t, true>());
    cudaFuncSetAttribute(k_scatter<uint64_t, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)scatter_smem<uint64_t, true>());
    done.push_back(dev);
}

template <typename KT, bool HAS_VAL>
fast_status sort_impl(fast_ctx *c, uint32_t nseg, uint64_t len, const KT *keys_in, const uint32_t *vals_in,
                      KT *ka, uint32_t *va, KT *kb, uint32_t *vb, uint32_t bit0, uint32_t bit1, KT **kout,
                      uint32_t **vout, cudaStream_t s, uint32_t *passes_out, Stations S = Stations{nullptr, 1},
                      uint64_t seg_max = 0) {
    const uint32_t npass = (bit1 - bit0 + 7) / 8;
    if (passes_out) *passes_out = npass;
    if (len == 0 || nseg == 0 || npass == 0) {
        *kout = const_cast<KT *>(keys_in);
        if (vout) *vout = const_cast<uint32_t *>(vals_in);
        return FAST_OK;
    }
    const uint64_t nch64 = ((S.nst > 1 ? seg_max : len) + kChunk - 1) / kChunk;
    if (nch64 > 0x7fffffffull) return set_error(c, FAST_EINVAL, "sort: segment too long");
    const uint32_t nchunks = (uint32_t)nch64;
    const size_t entries = (size_t)nseg * kRadix * nchunks;
    uint32_t *counts = nullptr;
    uint64_t *offs = nullptr;
    fast_status st;
    if ((st = dalloc_t(c, &counts, entries, s))) return st;
    if ((st = dalloc_t(c, &offs, entries, s))) {
        dfree(c, counts, entries * 4, s);
        return st;
    }
    const KT *src_k = keys_in;
    const uint32_t *src_v = vals_in;
    dim3 grid(nchunks, nseg);
    scatter_attrs();
    for (uint32_t pass = 0; pass < npass; pass++) {
        const uint32_t shift = bit0 + 8 * pass;
        KT *dk = (pass & 1) ? kb : ka;
        uint32_t *dv = (pass & 1) ? vb : va;
        k_hist<KT><<<grid, kThreads, 0, s>>>(src_k, len, nchunks, shift, counts, S), FAST_LAUNCHED(c);
        if ((st = scan_excl(c, counts, offs, (uint64_t)kRadix * nchunks, nseg, nullptr, s))) break;
        if (HAS_VAL && pass == 0 && src_v == nullptr)
            k_scatter<KT, true, true><<<grid, kThreads, scatter_smem<KT, true>(), s>>>(
                src_k, nullptr, dk, dv, len, nchunks, shift, counts, offs, S), FAST_LAUNCHED(c);
        else if (HAS_VAL)
            k_scatter<KT, true, false><<<grid, kThreads, scatter_smem<KT, true>(), s>>>(
                src_k, src_v, dk, dv, len, nchunks, shift, counts, offs, S), FAST_LAUNCHED(c);
        else
            k_scatter<KT, false, false><<<grid, kThreads, scatter_smem<KT, false>(), s>>>(
                src_k, nullptr, dk, nullptr, len, nchunks, shift, counts, offs, S), FAST_LAUNCHED(c);
        src_k = dk;
        src_v = dv;
    }
    dfree(c, counts, entries * 4, s);
    dfree(c, offs, entries * 8, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(c, e, "radix sort");
    *kout = const_cast<KT *>(src_k);
    if (vout) *vout = const_cast<uint32_t *>(src_v);
    return FAST_OK;
}

}  // namespace

fast_status sort_u32(fast_ctx *c, uint32_t nseg, uint64_t len, const uint32_t *keys_in, const uint32_t *vals_in,
                     uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, uint32_t bit0,
                     uint32_t bit1, uint32_t **keys_out, uint32_t **vals_out, cudaStream_t s, uint32_t *passes,
                     Stations S, uint64_t seg_max) {
    if (S.nst > 1 && (uint64_t)nseg * S.nst > 65535) return set_error(c, FAST_EINVAL, "sort: too many segments");
    return sort_impl<uint32_t, true>(c, S.nst > 1 ? nseg * S.nst : nseg, len, keys_in, vals_in, keys_a, vals_a,
                                     keys_b, vals_b, bit0, bit1, keys_out, vals_out, s, passes, S, seg_max);
}

fast_status sort_u64(fast_ctx *c, uint64_t len, uint64_t *keys_a, uint64_t *keys_b, uint32_t bit0, uint32_t bit1,
                     uint64_t **keys_out, cudaStream_t s) {
    // keys start in keys_a; passes alternate b, a, b, ...
    uint64_t *out = nullptr;
    fast_status st = sort_impl<uint64_t, false>(c, 1, len, keys_a, nullptr, keys_b, nullptr, keys_a, nullptr, bit0,
                                                bit1, &out, nullptr, s, nullptr);
    *keys_out = out;
    return st;
}

}  // namespace fastgb

namespace fastgb {
// ---------------------------------------------------------------------------
// fast_table_sort_static: one table's stable (key, id) sort with no device
// allocation.  Its scratch -- one ping-pong pair of keys and ids plus the
// per-chunk digit counts and offsets -- lives in the file-scope array below,
// sized for kStaticMaxKeys keys.  Every GPU that loads this library holds the
// array until the process exits; all calls on a device share it.
// ---------------------------------------------------------------------------

namespace {

constexpr uint64_t kStaticMaxKeys = 1ull << 20;
constexpr uint64_t kStaticChunks = (kStaticMaxKeys + kChunk - 1) / kChunk;
constexpr size_t kStaticCountsBytes = (size_t)kRadix * kStaticChunks * 4;
constexpr size_t kStaticOffsetsBytes = (size_t)kRadix * kStaticChunks * 8;
constexpr size_t kStaticBytes = kStaticMaxKeys * 4 * 2 + kStaticCountsBytes + kStaticOffsetsBytes;

static __device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself: it names a host stand-in).
cudaError_t scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace fastgb

extern "C" fast_status fast_table_sort_static(const uint32_t *d_keys, uint64_t n, uint32_t *d_skey, uint32_t *d_sid,
                                              void *stream) {
    using namespace fastgb;
    if (n > kStaticMaxKeys) return FAST_EINVAL;
    if (n == 0) return FAST_OK;
    if (!d_keys || !d_skey || !d_sid) return FAST_EINVAL;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_for_current_device(&base);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FAST_ECUDA;
    }
    uint32_t *tmp_k = reinterpret_cast<uint32_t *>(base);
    uint32_t *tmp_v = tmp_k + kStaticMaxKeys;
    uint32_t *counts = reinterpret_cast<uint32_t *>(base + kStaticMaxKeys * 8);
    uint64_t *offs = reinterpret_cast<uint64_t *>(base + kStaticMaxKeys * 8 + kStaticCountsBytes);
    // an error left pending by earlier work of the caller is reported (and
    // left in place for the caller) before anything is launched, so that the
    // check after the launches below sees only this call's own launch errors
    if (cudaPeekAtLastError() != cudaSuccess) return FAST_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t nchunks = (uint32_t)((n + kChunk - 1) / kChunk);
    const dim3 grid(nchunks, 1);
    scatter_attrs();
    // four 8-bit passes: keys -> scratch -> out -> scratch -> out
    const uint32_t *src_k = d_keys, *src_v = nullptr;
    for (uint32_t pass = 0; pass < 4; pass++) {
        uint32_t *dk = (pass & 1) ? d_skey : tmp_k;
        uint32_t *dv = (pass & 1) ? d_sid : tmp_v;
        const uint32_t shift = 8 * pass;
        k_hist<uint32_t><<<grid, kThreads, 0, s>>>(src_k, n, nchunks, shift, counts);
        k_scan<<<1, 1024, 0, s>>>(counts, offs, nchunks);
        if (pass == 0)
            k_scatter<uint32_t, true, true><<<grid, kThreads, scatter_smem<uint32_t, true>(), s>>>(
                src_k, nullptr, dk, dv, n, nchunks, shift, counts, offs);
        else
            k_scatter<uint32_t, true, false><<<grid, kThreads, scatter_smem<uint32_t, true>(), s>>>(
                src_k, src_v, dk, dv, n, nchunks, shift, counts, offs);
        src_k = dk;
        src_v = dv;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? FAST_OK : FAST_ECUDA;
}
