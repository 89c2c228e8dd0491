// k_sig.cu -- hash signature generation (§6.1 "Hash signature generation",
// §6.2 Min-Max hash, Algorithm 1).
//
// For each fingerprint S (K set bits of D) and hash function f, MinHash needs
// min_{x in S} h_f(x) and Min-Max hash also max_{x in S} h_f(x); the r values
// of table t are folded into one 32-bit bucket key (hash_combine).
//
// GB300 design.  Algorithm 1 evaluates h_f on every set bit (K*F evaluations
// per fingerprint).  Here the per-function ranking of [0, D) by h_f is built
// once per context ("hash mappings", Algorithm 1's single_hash, sorted); the
// minimum of h_f over S is then h_f of the first element of that ranking that
// lies in S -- the paper's own definition of MinHash as the first non-zero
// element under a permutation (§6.1) -- and the maximum is the first one from
// the other end.  A CTA takes a tile of 32 fingerprints and transposes them
// into a shared-memory bitmap M[x] (bit q set iff fingerprint q has bit x), so
// one lookup of M[x] tests x against all 32 fingerprints at once.  Each lane
// walks one (function, direction) ranking until every fingerprint of the tile
// has been hit; with K/D = 400/8192 that is ~80 steps instead of 400 hash
// evaluations per fingerprint.  Walks are handed out dynamically so lanes do
// not wait for each other.  The result is bit-identical to evaluating every
// element: it is the same minimum / maximum value.
//
// A direct-evaluation kernel covers shapes where the walk does not pay
// (K^2 < D) or does not fit shared memory.
#include <algorithm>

#include "fast_internal.cuh"

namespace fastgb {

namespace {

constexpr int kSigThreads = 448;  // 14 warps: 400 Min-Max walks keep most lanes busy (measured faster than 512)
constexpr int kTile = 32;

// Rank tables: walk[w][k], w = f (MinHash) or 2f / 2f+1 (Min-Max min / max),
// is the k-th element of [0, D) in ascending (min) or descending (max) order
// of h_f, ties broken by x.  Rows are padded to Dpad (multiple of 8) by
// repeating the last element, which can never produce a new hit.
__global__ void k_walk_build(const uint64_t *__restrict__ ha, const uint64_t *__restrict__ hb, uint32_t D,
                             uint32_t P2, uint32_t Dpad, int minmax, uint16_t *__restrict__ walk) {
    extern __shared__ uint64_t s_key[];
    const uint32_t f = blockIdx.x;
    const uint64_t a = ha[f], b = hb[f];
    const uint32_t a_lo = (uint32_t)a, a_hi = (uint32_t)(a >> 32);
    for (uint32_t x = threadIdx.x; x < P2; x += blockDim.x)
        s_key[x] = x < D ? ((uint64_t)hash_ab(a_lo, a_hi, b, x) << 16 | x) : ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= P2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < P2 / 2; i += blockDim.x) {
                uint32_t lo = 2 * i - (i & (stride - 1));
                uint32_t hi = lo + stride;
                bool asc = (lo & size) == 0;
                uint64_t x = s_key[lo], y = s_key[hi];
                if ((x > y) == asc) {
                    s_key[lo] = y;
                    s_key[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t k = threadIdx.x; k < Dpad; k += blockDim.x) {
        uint32_t kk = k < D ? k : D - 1;
        uint16_t xmin = (uint16_t)(s_key[kk] & 0xFFFF);
        if (minmax) {
            walk[(size_t)(2 * f) * Dpad + k] = xmin;
            walk[(size_t)(2 * f + 1) * Dpad + k] = (uint16_t)(s_key[D - 1 - kk] & 0xFFFF);
        } else {
            walk[(size_t)f * Dpad + k] = xmin;
        }
    }
}

__device__ __forceinline__ uint32_t u16_of(const uint4 &v, int s) {
    uint32_t w = s < 2 ? v.x : s < 4 ? v.y : s < 6 ? v.z : v.w;
    return (s & 1) ? (w >> 16) : (w & 0xFFFF);
}

// Signature kernel, walk variant.  Persistent CTAs loop over tiles of 32
// fingerprints.  Shared memory: M[D] masks and, per fingerprint and walk, the
// element x where the walk first hit it (16 bits; its hash value is computed
// once, in the combine step).  The walks are latency-bound chains of
// dependent loads, so the small footprint buys resident CTAs: three per SM.
template <bool MINMAX>
__global__ void __launch_bounds__(kSigThreads, 3)
    k_sig_walk(const uint16_t *__restrict__ idx, uint64_t N, uint32_t ld, uint32_t D, uint32_t K,
               const uint16_t *__restrict__ walk, uint32_t Dpad, uint32_t W, const uint64_t *__restrict__ ha,
               const uint64_t *__restrict__ hb, const uint64_t *__restrict__ zinit, uint32_t nb, uint32_t r,
               uint32_t *__restrict__ sig, uint64_t Nst, uint32_t *err, int vec16) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t next_walk;
    uint32_t *M = smem;
    const uint32_t Wp = W | 1u;  // odd row stride
    uint16_t *vals = reinterpret_cast<uint16_t *>(smem + ((D + 3) & ~3u));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t ntiles = (N + kTile - 1) / kTile;
    const uint32_t nk8 = Dpad / 8;

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = tile * kTile;
        const uint32_t nvalid = (uint32_t)(N - base < (uint64_t)kTile ? N - base : (uint64_t)kTile);
        for (uint32_t i = threadIdx.x; i < D; i += blockDim.x) M[i] = 0;
        if (threadIdx.x == 0) next_walk = 0;
        __syncthreads();

        // 1. transpose the tile into membership masks
        bool bad = false;
        for (uint32_t q = warp; q < nvalid; q += nwarps) {
            const uint16_t *row = idx + (base + q) * (uint64_t)ld;
            const uint32_t bit = 1u << q;
            if (vec16) {
                const uint4 *row4 = reinterpret_cast<const uint4 *>(row);
                for (uint32_t c = lane; c < (K + 7) / 8; c += 32) {
                    uint4 v = __ldg(row4 + c);
#pragma unroll
                    for (int s = 0; s < 8; s++) {
                        uint32_t k = c * 8 + s, x = u16_of(v, s);
                        if (k < K) {
                            if (x < D) atomicOr(&M[x], bit);
                            else bad = true;
                        }
                    }
                }
            } else {
                for (uint32_t k = lane; k < K; k += 32) {
                    uint32_t x = __ldg(row + k);
                    if (x < D) atomicOr(&M[x], bit);
                    else bad = true;
                }
            }
        }
        if (bad) set_err(err, ERR_BAD_INDEX);
        __syncthreads();

        // 2. walks: lane-private state, walks handed out one at a time
        const uint32_t done_mask = nvalid == 32 ? 0u : (~0u << nvalid);
        uint32_t w = atomicAdd(&next_walk, 1u);
        uint32_t found = done_mask, k8 = 0;
        const uint4 *seq = w < W ? reinterpret_cast<const uint4 *>(walk + (size_t)w * Dpad) : nullptr;
        uint4 nxt = w < W ? __ldg(seq) : make_uint4(0, 0, 0, 0);
        while (w < W) {
            const uint4 v = nxt;
            if (k8 + 1 < nk8) nxt = __ldg(seq + k8 + 1);  // next 8 steps in flight while these run
#pragma unroll
            for (int s = 0; s < 8; s++) {
                uint32_t x = u16_of(v, s);
                uint32_t m = M[x] & ~found;
                if (m) {
                    found |= m;
                    do {
                        uint32_t q = __ffs(m) - 1;
                        vals[q * Wp + w] = (uint16_t)x;
                        m &= m - 1;
                    } while (m);
                }
            }
            ++k8;
            if (found == ~0u || k8 >= nk8) {
                if (found != ~0u) set_err(err, ERR_WALK);
                w = atomicAdd(&next_walk, 1u);
                found = done_mask;
                k8 = 0;
                if (w < W) {
                    seq = reinterpret_cast<const uint4 *>(walk + (size_t)w * Dpad);
                    nxt = __ldg(seq);
                }
            }
        }
        __syncthreads();

        // 3. hash_combine: key of (fingerprint q = lane, table t)
        if ((uint32_t)lane < nvalid) {
            const uint32_t q = lane;
            for (uint32_t t = warp; t < nb; t += nwarps) {
                uint64_t z = __ldg(zinit + t);
                const uint32_t qf = MINMAX ? (r + 1) / 2 : r;
                for (uint32_t c = 0; c < r; c++) {
                    const uint32_t f = MINMAX ? t * qf + c / 2 : t * r + c;
                    const uint32_t x = vals[q * Wp + (MINMAX ? 2 * f + (c & 1) : f)];
                    const uint64_t a = __ldg(ha + f);
                    const uint32_t h = hash_ab((uint32_t)a, (uint32_t)(a >> 32), __ldg(hb + f), x);
                    z = mix64(z ^ (uint64_t)h);
                }
                sig[(uint64_t)t * Nst + base + q] = (uint32_t)(z >> 32);
            }
        }
        __syncthreads();
    }
}

// Signature kernel, direct variant: one CTA per fingerprint, one thread per
// table, every set bit hashed by every function of the table.
template <bool MINMAX>
__global__ void k_sig_direct(const uint16_t *__restrict__ idx, uint64_t N, uint32_t ld, uint32_t D, uint32_t K,
                             const uint64_t *__restrict__ ha, const uint64_t *__restrict__ hb,
                             const uint64_t *__restrict__ zinit, uint32_t nb, uint32_t r, uint32_t *__restrict__ sig,
                             uint64_t Nst, uint32_t *err) {
    for (uint64_t i = blockIdx.x; i < N; i += gridDim.x) {
        const uint16_t *row = idx + i * (uint64_t)ld;
        for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x) {
            uint64_t z = __ldg(zinit + t);
            const uint32_t nf = MINMAX ? (r + 1) / 2 : r;
            uint32_t c = 0;
            for (uint32_t g = 0; g < nf; g++) {
                uint32_t f = t * nf + g;
                uint64_t a = __ldg(ha + f), b = __ldg(hb + f);
                uint32_t lo = 0xFFFFFFFFu, hi = 0;
                for (uint32_t k = 0; k < K; k++) {
                    uint32_t x = __ldg(row + k);
                    if (x >= D) {
                        set_err(err, ERR_BAD_INDEX);
                        x = 0;
                    }
                    uint32_t h = hash_ab((uint32_t)a, (uint32_t)(a >> 32), b, x);
                    lo = min(lo, h);
                    hi = max(hi, h);
                }
                z = mix64(z ^ (uint64_t)lo);
                ++c;
                if (MINMAX && c < r) {
                    z = mix64(z ^ (uint64_t)hi);
                    ++c;
                }
            }
            sig[(uint64_t)t * Nst + i] = (uint32_t)(z >> 32);
        }
    }
}

size_t walk_smem(const fast_ctx *c) {
    return (size_t)((c->p.D + 3) & ~3u) * 4 + (((size_t)kTile * (c->W | 1u) * 2 + 15) & ~(size_t)15);
}

}  // namespace

fast_status sig_setup(fast_ctx *c) {
    const fast_params &p = c->p;
    c->F = p.kind == FAST_MINHASH ? p.b * p.r : p.b * ((p.r + 1) / 2);
    c->W = p.kind == FAST_MINHASH ? c->F : 2 * c->F;
    std::vector<uint64_t> a(c->F), b(c->F), z(p.b);
    for (uint32_t f = 0; f < c->F; f++) {
        a[f] = sm64(p.seed, 2ull * f) | 1ull;
        b[f] = sm64(p.seed, 2ull * f + 1);
    }
    for (uint32_t t = 0; t < p.b; t++) z[t] = sm64(p.seed, 2ull * c->F + t);
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_a, 8 * c->F)) || (e = cudaMalloc(&c->d_b, 8 * c->F)) ||
        (e = cudaMalloc(&c->d_zinit, 8 * p.b)))
        return cuda_fail(c, e, "sig_setup alloc");
    cudaMemcpy(c->d_a, a.data(), 8 * c->F, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_b, b.data(), 8 * c->F, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_zinit, z.data(), 8 * p.b, cudaMemcpyHostToDevice);

    // The walk pays when the expected walk length ~4 D/K per tile beats K
    // evaluations per fingerprint, i.e. roughly K^2 >= D; it also needs the
    // masks and results to fit shared memory.
    c->Dpad = (p.D + 7) & ~7u;
    c->use_walk = (uint64_t)p.K * p.K >= p.D && p.D <= 16384 && walk_smem(c) <= 200 * 1024;
    if (!c->use_walk) return FAST_OK;
    uint32_t P2 = 1;
    while (P2 < p.D) P2 <<= 1;
    if ((e = cudaMalloc(&c->d_walk, (size_t)c->W * c->Dpad * 2))) return cuda_fail(c, e, "walk alloc");
    size_t sm = (size_t)P2 * 8;
    cudaFuncSetAttribute(k_walk_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_walk_build<<<c->F, 1024, sm>>>(c->d_a, c->d_b, p.D, P2, c->Dpad, p.kind == FAST_MINMAX, c->d_walk), FAST_LAUNCHED(c);
    if ((e = cudaGetLastError())) return cuda_fail(c, e, "k_walk_build");
    if ((e = cudaDeviceSynchronize())) return cuda_fail(c, e, "k_walk_build sync");
    size_t sms = walk_smem(c);
    if (p.kind == FAST_MINMAX)
        cudaFuncSetAttribute(k_sig_walk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
    else
        cudaFuncSetAttribute(k_sig_walk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
    return FAST_OK;
}

fast_status sig_launch_rows(fast_ctx *c, const uint16_t *d_idx, uint64_t N, uint32_t ld, uint32_t *d_sig, uint64_t Nst,
                            cudaStream_t s) {
    if (N == 0) return FAST_OK;
    const fast_params &p = c->p;
    const bool mm = p.kind == FAST_MINMAX;
    if (c->use_walk) {
        uint64_t ntiles = (N + kTile - 1) / kTile;
        int vec16 = (ld % 8 == 0) && ((uintptr_t)d_idx % 16 == 0);
        size_t sms = walk_smem(c);
        int per_sm = 0;
        if (mm)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sig_walk<true>, kSigThreads, sms);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sig_walk<false>, kSigThreads, sms);
        uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)c->num_sms * std::max(per_sm, 1));
        if (mm)
            k_sig_walk<true><<<(unsigned)grid, kSigThreads, sms, s>>>(d_idx, N, ld, p.D, p.K, c->d_walk, c->Dpad,
                                                                      c->W, c->d_a, c->d_b, c->d_zinit, p.b, p.r,
                                                                      d_sig, Nst, c->d_err, vec16), FAST_LAUNCHED(c);
        else
            k_sig_walk<false><<<(unsigned)grid, kSigThreads, sms, s>>>(d_idx, N, ld, p.D, p.K, c->d_walk, c->Dpad,
                                                                       c->W, c->d_a, c->d_b, c->d_zinit, p.b, p.r,
                                                                       d_sig, Nst, c->d_err, vec16), FAST_LAUNCHED(c);
    } else {
        unsigned grid = (unsigned)std::min<uint64_t>(N, (uint64_t)c->num_sms * 16);
        unsigned thr = std::min<uint32_t>(256, (p.b + 31) & ~31u);
        if (mm)
            k_sig_direct<true><<<grid, thr, 0, s>>>(d_idx, N, ld, p.D, p.K, c->d_a, c->d_b, c->d_zinit, p.b, p.r,
                                                    d_sig, Nst, c->d_err), FAST_LAUNCHED(c);
        else
            k_sig_direct<false><<<grid, thr, 0, s>>>(d_idx, N, ld, p.D, p.K, c->d_a, c->d_b, c->d_zinit, p.b, p.r,
                                                     d_sig, Nst, c->d_err), FAST_LAUNCHED(c);
    }
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(c, e, "sig kernel") : FAST_OK;
}

fast_status sig_launch(fast_ctx *c, const uint16_t *d_idx, uint64_t N, uint32_t ld, uint32_t *d_sig,
                       cudaStream_t s) {
    return sig_launch_rows(c, d_idx, N, ld, d_sig, N, s);
}

}  // namespace fastgb
