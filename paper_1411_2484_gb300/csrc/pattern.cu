// pattern.cu -- the full-period D-dimensional pattern of one 32-bit instance
// by enumeration (the O(p L0) method that follows Eq. 7 in the paper).
//
// Over the full period n(p-1), the ciphertext value c0 occurs p-1 times, once
// with each skip s = s_(k+1) in (Z/pZ)*, and always with the message
// m = c0^d mod n (Eq. 2).  So the D-tuples (c0, c_(k+1), ..., c_(k+D-1)) of the
// whole period with c0 in a range [c_lo, c_lo + L0) are the points
//     c_(k+j) = (m + s + a s + ... + a^(j-1) s)^e mod n   (skips mod p, sum mod n)
// for every c0 of the range and every s -- L0 (p-1) exponentiation chains
// instead of a walk over n(p-1) numbers.  A thread takes NPT consecutive
// skips of one c0 and runs them as NPT independent chains of the same
// exponent program (gencore.cuh); each point adds one to a histogram of
// nb^(D-1) counters (bin floor(c / L1) per coordinate, L1 = ceil(n / nb)).
#include <cuda_runtime.h>

#include "gencore.cuh"

namespace phprng {

// floor(x / L1) for L1 >= 2: with r = floor(2^32 / L1) the estimate
// floor(x r / 2^32) is the quotient or one below it (r is short of 2^32 / L1 by
// less than 1 and x < 2^32), and one comparison decides.
__device__ __forceinline__ uint32_t div_by_width(uint32_t x, uint32_t L1, uint32_t r)
{
    uint32_t q = umulhi32(x, r);
    if ((uint64_t)(q + 1) * L1 <= x) ++q;
    return q;
}

// SMEM: histograms of at most kSmemBins counters are gathered per block in
// shared memory and added to the device counters once (few, hot counters
// would otherwise serialise the device-wide reductions).
static constexpr uint32_t kSmemBins = 8192;

// The counts go to 32-bit counters (nb^(D-1) <= 2^24: at most 64 MiB, which
// L2 holds, where 64-bit counters spilled their reductions to DRAM); the
// host runs chunks of c0 with fewer than 2^32 points each and folds the
// 32-bit counters into the caller's 64-bit ones after every chunk.
template <int NPT, bool SMEM>
__global__ void __launch_bounds__(256, 2)
pattern_kernel(DevInst P, ExpProg pg, SkipConst sk, const uint32_t *__restrict__ mtab, uint64_t L0,
               int D, uint32_t nb, uint32_t L1, uint32_t rL1, uint64_t lim, uint32_t bins,
               unsigned int *__restrict__ hist)
{
    extern __shared__ unsigned int sh[];
    if (SMEM) {
        for (uint32_t k = threadIdx.x; k < bins; k += blockDim.x) sh[k] = 0;
        __syncthreads();
    }
    const uint32_t p = sk.p, n = (uint32_t)P.n;
    const uint64_t per_c0 = (p - 2 + NPT) / NPT;          // thread items per c0: skips 1 .. p-1
    const uint64_t items = L0 * per_c0;
    // item it = q per_c0 + r; the grid stride advances (q, r) without a
    // division per item (one per thread here)
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t it0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t dq = stride / per_c0, dr = stride - dq * per_c0;
    uint64_t q = it0 / per_c0, r = it0 - q * per_c0;
    for (uint64_t it = it0; it < items; it += stride) {
        const uint32_t s0 = (uint32_t)(r * NPT) + 1;
        const uint32_t m = mtab[q];
        uint32_t t[NPT], acc[NPT], x[NPT], idx[NPT];
        bool inside[NPT];
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            // skips past p-1 (the last item of a c0) are computed and not counted
            t[u] = s0 + u < p ? s0 + u : 1u;
            acc[u] = m;
            idx[u] = 0;
            inside[u] = s0 + u < p;
        }
        uint32_t scale = 1;
        for (int j = 1; j < D; ++j) {
#pragma unroll
            for (int u = 0; u < NPT; ++u) acc[u] = addmod32(acc[u], t[u], n);
            encrypt<NPT, uint32_t>(P, pg, acc, x);                     // Eq. 9c
#pragma unroll
            for (int u = 0; u < NPT; ++u) {
                idx[u] += (L1 == 1 ? x[u] : div_by_width(x[u], L1, rL1)) * scale;
                inside[u] = inside[u] && x[u] < lim;                    // region [0, nb L1)
            }
            scale *= nb;
            if (j + 1 < D) {
#pragma unroll
                for (int u = 0; u < NPT; ++u) t[u] = mont32(t[u], sk.aM, p, sk.pinv);   // Eq. 9a
            }
        }
#pragma unroll
        for (int u = 0; u < NPT; ++u)
            if (inside[u]) atomicAdd((SMEM ? sh : hist) + idx[u], 1u);
        q += dq;
        r += dr;
        if (r >= per_c0) {
            r -= per_c0;
            ++q;
        }
    }
    if (SMEM) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < bins; k += blockDim.x)
            if (sh[k]) atomicAdd(hist + k, sh[k]);
    }
}

// hist64[i] += hist32[i]; hist32[i] = 0.
__global__ void __launch_bounds__(256)
fold_counts_kernel(unsigned int *__restrict__ h32, unsigned long long *__restrict__ h64, uint64_t bins)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < bins;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned int v = h32[i];
        if (v) {
            h64[i] += v;
            h32[i] = 0;
        }
    }
}

// The constant-skip generator (s_k = b; b = 1 is the unit skip, counter mode)
// has period n and meets each c0 once, with message m = c0^d mod n, so its
// full-period pattern has one point per c0: c_(k+j) = (m + j b)^e mod n.  A
// thread takes NPT consecutive c0, decrypts them with the program of d
// (Pd, pgd) and encrypts the D-1 successors with the program of e.
template <int NPT, bool SMEM>
__global__ void __launch_bounds__(256, 2)
pattern_const_kernel(DevInst P, ExpProg pg, DevInst Pd, ExpProg pgd, uint32_t b, uint64_t c_lo,
                     uint64_t L0, int D, uint32_t nb, uint32_t L1, uint32_t rL1, uint64_t lim, uint32_t bins,
                     unsigned long long *__restrict__ hist)
{
    extern __shared__ unsigned int sh[];
    if (SMEM) {
        for (uint32_t k = threadIdx.x; k < bins; k += blockDim.x) sh[k] = 0;
        __syncthreads();
    }
    const uint32_t n = (uint32_t)P.n;
    const uint64_t items = (L0 + NPT - 1) / NPT;
    for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q0 = it * NPT;
        uint32_t c0[NPT], m[NPT], acc[NPT], x[NPT], idx[NPT];
        bool inside[NPT];
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            c0[u] = (uint32_t)(c_lo + (q0 + u < L0 ? q0 + u : 0));   // past L0: computed, not counted
            idx[u] = 0;
            inside[u] = q0 + u < L0;
        }
        encrypt<NPT, uint32_t>(Pd, pgd, c0, m);                       // m = c0^d (Eq. 2)
        uint32_t scale = 1;
#pragma unroll
        for (int u = 0; u < NPT; ++u) acc[u] = m[u];
        for (int j = 1; j < D; ++j) {
#pragma unroll
            for (int u = 0; u < NPT; ++u) acc[u] = addmod32(acc[u], b, n);
            encrypt<NPT, uint32_t>(P, pg, acc, x);                      // Eq. 9c
#pragma unroll
            for (int u = 0; u < NPT; ++u) {
                idx[u] += (L1 == 1 ? x[u] : div_by_width(x[u], L1, rL1)) * scale;
                inside[u] = inside[u] && x[u] < lim;                    // region [0, nb L1)
            }
            scale *= nb;
        }
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            if (!inside[u]) continue;
            if (SMEM)
                atomicAdd(sh + idx[u], 1u);
            else
                atomicAdd(hist + idx[u], 1ull);
        }
    }
    if (SMEM) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < bins; k += blockDim.x)
            if (sh[k]) atomicAdd(hist + k, (unsigned long long)sh[k]);
    }
}

int launch_pattern_const(const DevInst &P, const ExpProg &pg, const DevInst &Pd, const ExpProg &pgd,
                         uint32_t b, uint64_t c_lo, uint64_t L0, int D, uint32_t nb, uint32_t L1r,
                         uint64_t *hist, void *stream, std::string *err)
{
    constexpr int NPT = 8;
    const uint32_t n = (uint32_t)P.n;
    const uint32_t L1 = L1r ? L1r : (uint32_t)((n + (uint64_t)nb - 1) / nb);
    const uint64_t lim = (uint64_t)nb * L1;                 // >= n for the whole range
    const uint32_t rL1 = L1 >= 2 ? (uint32_t)((1ull << 32) / L1) : 0u;
    uint32_t bins = 1;
    for (int d = 1; d < D; ++d) bins *= nb;
    const bool smem = bins <= kSmemBins;
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &bps, smem ? pattern_const_kernel<NPT, true> : pattern_const_kernel<NPT, false>, 256,
        smem ? kSmemBins * 4 : 0);
    const uint64_t items = (L0 + NPT - 1) / NPT;
    uint64_t grid = (items + 255) / 256;
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * (bps > 0 ? bps : 1) * 8;
    if (grid > cap) grid = cap;
    if (grid == 0) return PHPRNG_OK;
    if (smem)
        pattern_const_kernel<NPT, true><<<(unsigned)grid, 256, bins * 4, (cudaStream_t)stream>>>(
            P, pg, Pd, pgd, b, c_lo, L0, D, nb, L1, rL1, lim, bins, (unsigned long long *)hist);
    else
        pattern_const_kernel<NPT, false><<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(
            P, pg, Pd, pgd, b, c_lo, L0, D, nb, L1, rL1, lim, bins, (unsigned long long *)hist);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("pattern_const_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_pattern(const DevInst &P, const ExpProg &pg, const SkipConst &sk, const uint32_t *mtab,
                   uint64_t L0, int D, uint32_t nb, uint32_t L1r, uint64_t *hist, void *stream,
                   std::string *err)
{
    constexpr int NPT = 8;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)P.n;
    const uint32_t L1 = L1r ? L1r : (uint32_t)((n + (uint64_t)nb - 1) / nb);
    const uint64_t lim = (uint64_t)nb * L1;                 // >= n for the whole range
    const uint32_t rL1 = L1 >= 2 ? (uint32_t)((1ull << 32) / L1) : 0u;
    uint64_t bins = 1;
    for (int d = 1; d < D; ++d) bins *= nb;
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pattern_kernel<NPT, false>, 256, 0);
    const bool smem = bins <= kSmemBins;
    if (smem)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pattern_kernel<NPT, true>, 256, kSmemBins * 4);
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * (bps > 0 ? bps : 1) * 8;
    unsigned int *h32 = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&h32, bins * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h32, 0, bins * sizeof(unsigned int), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h32) cudaFreeAsync(h32, s);
        *err = std::string("pattern counters: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? PHPRNG_ENOMEM : PHPRNG_ECUDA;
    }
    // chunks of c0 with fewer than 2^32 points, so no 32-bit counter wraps
    const uint64_t per_c0 = sk.p - 1;
    const uint64_t chunk = ((1ull << 32) - 1) / per_c0 ? ((1ull << 32) - 1) / per_c0 : 1;
    const uint64_t fold_grid = (bins + 255) / 256 < cap ? (bins + 255) / 256 : cap;
    for (uint64_t q0 = 0; q0 < L0 && e == cudaSuccess; q0 += chunk) {
        const uint64_t lq = L0 - q0 < chunk ? L0 - q0 : chunk;
        const uint64_t items = lq * ((sk.p - 2 + NPT) / NPT);
        uint64_t grid = (items + 255) / 256;
        if (grid > cap) grid = cap;
        if (smem)
            pattern_kernel<NPT, true><<<(unsigned)grid, 256, bins * 4, s>>>(P, pg, sk, mtab + q0, lq, D, nb,
                                                                           L1, rL1, lim, (uint32_t)bins, h32);
        else
            pattern_kernel<NPT, false><<<(unsigned)grid, 256, 0, s>>>(P, pg, sk, mtab + q0, lq, D, nb, L1,
                                                                     rL1, lim, (uint32_t)bins, h32);
        fold_counts_kernel<<<(unsigned)fold_grid, 256, 0, s>>>(h32, (unsigned long long *)hist, bins);
        e = cudaGetLastError();
    }
    cudaFreeAsync(h32, s);
    if (e != cudaSuccess) {
        *err = std::string("pattern_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

}  // namespace phprng
