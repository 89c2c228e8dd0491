// k_scan.cu -- device-wide exclusive scan of uint32 counts into uint64
// offsets, for `nseg` equal segments at once (digit counts of every table in
// the radix sort, per-row counts of the detection list).
//
// Three launches, no inter-CTA waits: tile sums, a scan of the tile sums per
// segment, then every tile rescanned with its offset.  Each tile is 4096
// counts; a segment of n counts reads them twice and writes n offsets.
#include "fast_internal.cuh"

namespace fastgb {

namespace {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total.
template <typename T>
__device__ __forceinline__ T block_scan_excl(T x, T *wsum, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(~0u, v, d);
        if (lane >= d) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? wsum[lane] : (T)0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = __shfl_up_sync(~0u, w, d);
            if (lane >= d) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    T r = v - x + (warp ? wsum[warp - 1] : (T)0);
    *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t *__restrict__ in, uint64_t n, uint32_t nblk,
                                                          uint64_t *__restrict__ part) {
    __shared__ uint64_t wsum[32];
    const uint32_t seg = blockIdx.y, blk = blockIdx.x;
    const uint32_t *x = in + (uint64_t)seg * n;
    const uint64_t lo = (uint64_t)blk * kTile, hi = min(lo + kTile, n);
    uint64_t s = 0;
    for (uint64_t e = lo + threadIdx.x; e < hi; e += kThreads) s += x[e];
    uint64_t tot;
    block_scan_excl<uint64_t>(s, wsum, &tot);
    if (threadIdx.x == 0) part[(uint64_t)seg * nblk + blk] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_part(uint64_t *__restrict__ part, uint32_t nblk,
                                                    uint64_t *__restrict__ totals) {
    __shared__ uint64_t wsum[32];
    uint64_t *p = part + (uint64_t)blockIdx.x * nblk;
    uint64_t carry = 0;
    for (uint32_t base = 0; base < nblk; base += blockDim.x) {
        const uint32_t k = base + threadIdx.x;
        const uint64_t v = k < nblk ? p[k] : 0;
        uint64_t tot;
        const uint64_t ex = block_scan_excl<uint64_t>(v, wsum, &tot);
        if (k < nblk) p[k] = carry + ex;
        carry += tot;
    }
    if (totals && threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(const uint32_t *__restrict__ in, uint64_t *__restrict__ out,
                                                         uint64_t n, uint32_t nblk, const uint64_t *__restrict__ part) {
    __shared__ uint64_t wsum[32];
    const uint32_t seg = blockIdx.y, blk = blockIdx.x;
    const uint32_t *x = in + (uint64_t)seg * n;
    uint64_t *o = out + (uint64_t)seg * n;
    const uint64_t lo = (uint64_t)blk * kTile + (uint64_t)threadIdx.x * kItems;
    uint32_t v[kItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        v[k] = lo + k < n ? x[lo + k] : 0u;
        s += v[k];
    }
    uint64_t tot;
    uint64_t run = part[(uint64_t)seg * nblk + blk] + block_scan_excl<uint64_t>(s, wsum, &tot);
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        if (lo + k < n) o[lo + k] = run;
        run += v[k];
    }
}

}  // namespace

fast_status scan_excl(fast_ctx *c, const uint32_t *in, uint64_t *out, uint64_t n, uint32_t nseg, uint64_t *totals,
                      cudaStream_t s) {
    if (n == 0 || nseg == 0) {
        if (totals && nseg) cudaMemsetAsync(totals, 0, 8ull * nseg, s);
        return FAST_OK;
    }
    const uint64_t nb64 = (n + kTile - 1) / kTile;
    if (nb64 > 0x7fffffffull) return set_error(c, FAST_EINVAL, "scan: too long");
    const uint32_t nblk = (uint32_t)nb64;
    uint64_t *part = nullptr;
    fast_status st = dalloc_t(c, &part, (size_t)nblk * nseg, s);
    if (st) return st;
    const dim3 g(nblk, nseg);
    k_scan_reduce<<<g, kThreads, 0, s>>>(in, n, nblk, part), FAST_LAUNCHED(c);
    k_scan_part<<<nseg, 1024, 0, s>>>(part, nblk, totals), FAST_LAUNCHED(c);
    k_scan_apply<<<g, kThreads, 0, s>>>(in, out, n, nblk, part), FAST_LAUNCHED(c);
    dfree(c, part, (size_t)nblk * nseg * 8, s);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(c, e, "scan") : FAST_OK;
}

}  // namespace fastgb
