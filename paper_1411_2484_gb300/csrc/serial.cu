// serial.cu -- fused serial-test and poker-test consumers (Tests section,
// items 1-6: the one-dimensional frequency test, the two- to five-dimensional
// serial tests and the poker test) for 32-bit moduli.
//
// The numbers are generated exactly as by the plain kernels (gencore.cuh) and
// never stored: each one's bin floor(B R) is formed from integers, the
// stream's consecutive non-overlapping D-tuples of bins are assembled in
// shared memory (a tuple may span lanes and warp groups), and each tuple adds
// one to a histogram of B^D counters in device memory, pooled over the
// launch's streams.  B^D is at most 2^24, so the histogram (<= 128 MiB of
// 64-bit counters, 8 MiB at the paper's 2^20 bins) stays in or near L2 and
// the additions are L2 reductions.
#include <algorithm>
#include <cuda_runtime.h>

#include "gencore.cuh"

namespace phprng {

#ifndef PH_SERIAL_MINB
#define PH_SERIAL_MINB 3
#endif
#ifndef PH_SERIAL_WARPS
#define PH_SERIAL_WARPS 8
#endif
static constexpr int kSerialWarps = PH_SERIAL_WARPS;   // warps per block of serial_kernel (3 blocks per SM, exponent tables in shared memory)

// Per warp of the generating kernels below: the exponent program's table of up
// to kProg8MaxTable odd powers (NPT/4 16-byte rows per lane and entry; the
// launches run 8 numbers per lane), in dynamic shared memory after the
// kernel's static arrays.
static constexpr size_t kEtbWarpBytes = kProg8MaxTable * (8 / 4) * 32 * sizeof(uint4);
extern __shared__ uint4 g_etb[];

// Dynamic shared memory of a launch of `warps` warps (the kernel's limit is
// raised when it passes the default 48 KiB; current device).
template <typename K>
static size_t etb_smem(K kernel, int warps)
{
    const size_t bytes = (size_t)warps * kEtbWarpBytes;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return bytes;
}

// The bin of a number, floor(B R) taken on the double R = RN((c+1)/(n+1))
// (Eq. 9d) with one IEEE product, RN(R B), then truncation -- what a program
// binning the generator's doubles computes.  For n < 2^32 and B <= 2^20 this
// is the exact floor(B (c+1)/(n+1)) except when (c+1)/(n+1) is exactly k/B:
// otherwise B (c+1)/(n+1) is at least 1/(n+1) >= 2^-32 from an integer, while
// the two roundings move it by less than B 2^-52 <= 2^-32.  At an exact k/B
// the double product can land just below k (B = 100: k = 29, 57, 58, where
// RN(RN(k/100) 100) < k), so that case is decided by the double arithmetic
// itself.
//
// The exact bin from integers: with vN = (c+1) 2^(32-ybits) < yN and
// r = floor(B 2^32 / yN), floor(vN r / 2^32) is the bin or one below it (r is
// short of B 2^32 / yN by less than 1 and vN < 2^32), and one exact comparison
// decides.  The final remainder B vN - k yN lies in [0, yN), below 2^32, so it
// is zero exactly when its low word is, and that word comes from the two
// products of the comparison: lo(B vN) - lo((est+1) yN), plus yN when est was
// not raised.  A zero remainder -- an exact k/B, about 1 number in 2^31 at
// random -- sends the number to the double arithmetic.
__device__ __forceinline__ uint32_t serial_bin_int(uint32_t c, uint32_t yN, uint32_t ybits, uint32_t r,
                                                   uint32_t B, uint32_t *exact_multiple)
{
    const uint32_t vN = (c + 1) << (32 - ybits);
    uint32_t est = umulhi32(vN, r);
    const uint64_t P1 = (uint64_t)(est + 1) * yN, P2 = (uint64_t)vN * B;
    const bool up = P1 <= P2;
    est += up ? 1u : 0u;
    const uint32_t d = (uint32_t)P2 - (uint32_t)P1;
    *exact_multiple = d == (up ? 0u : 0u - yN) ? 1u : 0u;
    return est;
}

__device__ __forceinline__ uint32_t serial_bin_double(uint32_t c, uint32_t yN, uint32_t ybits, uint32_t B)
{
    const double R = __ddiv_rn((double)(c + 1), (double)(yN >> (32 - ybits)));
    return (uint32_t)__dmul_rn(R, (double)B);
}

__device__ __forceinline__ uint32_t serial_bin(uint32_t c, uint32_t yN, uint32_t ybits, uint32_t r,
                                               uint32_t B)
{
    uint32_t em;
    const uint32_t est = serial_bin_int(c, yN, ybits, r, B, &em);
    return em ? serial_bin_double(c, yN, ybits, B) : est;
}

// The bins of a lane's NPT numbers: the integer path for all of them without
// branches, then the double arithmetic for the exact multiples, in the rare
// lanes that have one.
template <int NPT, int C = (NPT % 4 == 0 ? 4 : NPT)>
__device__ __forceinline__ void serial_bins(const uint32_t (&x)[NPT], uint32_t yN, uint32_t ybits, uint32_t r,
                                            uint32_t B, uint32_t (&b)[NPT])
{
#pragma unroll
    for (int u0 = 0; u0 < NPT; u0 += C) {                // C numbers at a time (register pressure)
        uint32_t em = 0;
#pragma unroll
        for (int u = u0; u < u0 + C; ++u) {
            uint32_t e;
            b[u] = serial_bin_int(x[u], yN, ybits, r, B, &e);
            em |= e << u;
        }
        if (em) {
#pragma unroll
            for (int u = u0; u < u0 + C; ++u)
                if ((em >> u) & 1u) b[u] = serial_bin_double(x[u], yN, ybits, B);
        }
    }
}

// Poker category of five denominations: the sum over the cards of how many
// cards share the card's denomination is 5 (all different), 7 (one pair),
// 9 (two pairs), 11 (three of a kind), 13 (full house), 17 (four of a kind)
// or 25 (five of a kind), one value per category.
__device__ __forceinline__ uint32_t poker_category(const uint32_t *h)
{
    uint32_t sum = 0;
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) sum += h[a] == h[b] ? 1u : 0u;
    switch (sum) {
    case 5: return 0;
    case 7: return 1;
    case 9: return 2;
    case 11: return 3;
    case 13: return 4;
    case 17: return 5;
    default: return 6;
    }
}

// Shared counters of one warp: with POKER, 7 categories x 32 lanes, each lane
// counting its own hands (no atomics); otherwise the serial test's bins when
// there are at most kLocalBins of them, counted with shared atomics.  Either
// way they are added to the device histogram at the end of the call, and
// every 2^23 groups before that, so no 32-bit counter can overflow (a lane
// counts at most 2 hands of a 256-number group, a warp at most 256 tuples).
constexpr uint32_t kLocalBins = 7 * 32;
constexpr uint64_t kLocalFlushGroups = 1ull << 23;

template <bool POKER>
__device__ __forceinline__ void flush_local(uint32_t *cnt, uint32_t nbins, int lane,
                                            unsigned long long *hist)
{
    __syncwarp();
    if (POKER) {
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            uint32_t v = cnt[c * 32 + lane];
            cnt[c * 32 + lane] = 0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
            if (lane == 0 && v) atomicAdd(hist + c, (unsigned long long)v);
        }
    } else {
        for (uint32_t b = lane; b < nbins; b += 32) {
            const uint32_t v = cnt[b];
            cnt[b] = 0;
            if (v) atomicAdd(hist + b, (unsigned long long)v);
        }
    }
    __syncwarp();
}

// POKER: hands of five cards, denominations floor(10 R), into 7 category
// counters (D = 5, B = 10); otherwise the serial test's B^D counters.
template <int NPT, bool POKER, int WB>
__global__ void __launch_bounds__(WB * 32, PH_SERIAL_MINB)
serial_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog,
              const ExpProg8 *__restrict__ prog8, DevState st,
              SkipConst sk, uint64_t first, uint64_t num, uint64_t per_inst, int D, uint32_t B,
              unsigned long long *__restrict__ hist, const uint32_t *__restrict__ order)
{
    constexpr uint64_t G = 32 * NPT;
    __shared__ uint32_t tb[WB][32 * NPT + 8];  // per warp: a carried tuple start, then one group
    __shared__ uint32_t lc[WB][kLocalBins];         // per warp: shared counters (flush_local)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t w = (uint64_t)blockIdx.x * WB + warp;
    if (w >= num) return;
    const uint64_t j = order ? order[w] : w;
    const uint64_t i = first + j;
    const DevInst P = inst[i];
    const ExpProg &pg = prog[i];
    const ExpProg8 &pg8 = prog8[i];
    uint4 *etb = g_etb + warp * kProg8MaxTable * (NPT / 4) * 32;   // this warp's exponent table
    const uint32_t r = (uint32_t)(((uint64_t)B << 32) / P.yN);
    uint32_t nbins = 1;
    for (int d = 0; d < D && nbins <= kLocalBins; ++d) nbins *= B;
    const bool local = POKER || nbins <= kLocalBins;
    uint32_t *cnt = lc[warp];
    if (local)
        for (uint32_t b = lane; b < kLocalBins; b += 32) cnt[b] = 0;
    uint32_t M = (uint32_t)st.m[i];
    uint32_t sig = mont32((uint32_t)st.s[i], sk.lane[lane], sk.p, sk.pinv);
    const uint64_t pos_after = st.pos[i] + per_inst;
    uint32_t *buf = tb[warp];
    uint32_t carry = 0;                                   // bins waiting at buf[0 .. carry), < D
    uint32_t x[NPT], sig_last = sig;
    uint64_t g_last = 0;
    for (uint64_t g0 = 0; g0 < per_inst; g0 += G) {
        uint32_t sv[NPT], msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        messages32<NPT>(P, sk, lane, my0, per_inst, M, sig, sv, msg);
        encrypt32_p8<NPT>(P, pg, pg8, msg, x, etb, lane);
        {
            uint32_t b[NPT];
            serial_bins<NPT>(x, P.yN, P.ybits, r, B, b);
#pragma unroll
            for (int u = 0; u < NPT; ++u)
                if (my0 + u < per_inst) buf[carry + NPT * lane + u] = b[u];
        }
        __syncwarp();
        const uint32_t valid = per_inst - g0 < G ? (uint32_t)(per_inst - g0) : (uint32_t)G;
        const uint32_t total = carry + valid, ntup = total / (uint32_t)D;
        for (uint32_t t = lane; t < ntup; t += 32) {
            if constexpr (POKER) {
                cnt[poker_category(buf + t * 5) * 32 + lane] += 1u;
            } else {
                uint32_t idx = 0, scale = 1;
                for (int d = 0; d < D; ++d) {
                    idx += buf[t * D + d] * scale;
                    scale *= B;
                }
                if (local)
                    atomicAdd(cnt + idx, 1u);
                else
                    atomicAdd(hist + idx, 1ull);
            }
        }
        if (local && (g0 / G) % kLocalFlushGroups == kLocalFlushGroups - 1)
            flush_local<POKER>(cnt, nbins, lane, hist);
        const uint32_t rem = total - ntup * (uint32_t)D;
        const uint32_t keep = (uint32_t)lane < rem ? buf[ntup * D + lane] : 0u;
        __syncwarp();
        if ((uint32_t)lane < rem) buf[lane] = keep;
        __syncwarp();
        carry = rem;
    }
    if (local) flush_local<POKER>(cnt, nbins, lane, hist);
    write_state_after<NPT, uint32_t, uint32_t>(st, sk, i, lane, g_last, per_inst, pos_after, M, sig_last,
                                               x);
}

// Runs test (Tests section): bits b_k = (R_k > 1/2), i.e. c > (n-1)/2 (R is
// exactly 1/2 only for c = (n-1)/2, and no rounding crosses 1/2 since a
// nonzero distance to it is at least 1/(2(n+1))).  Per warp group the 256
// bits go to shared memory as 8 words (number k at bit k % 32 of word k / 32)
// with the transition words T (T_k = b_k != b_(k-1); T_0 against the bit of the
// run still open from the previous group).  A run ends at k when T_(k+1) is
// set; its start is the highest transition at or below k, or, when there is
// none, it began in an earlier group and adds the carried length.  The run
// still open at the group's end is carried; the one open at the call's end is
// not counted.  Counts go to a per-warp shared histogram, flushed at the end.
template <int NPT>
__global__ void __launch_bounds__(256, PH_SERIAL_MINB)
runs_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog,
            const ExpProg8 *__restrict__ prog8, DevState st,
            SkipConst sk, uint64_t first, uint64_t num, uint64_t per_inst, int lmax,
            unsigned long long *__restrict__ hist, const uint32_t *__restrict__ order)
{
    constexpr uint64_t G = 32 * NPT;
    constexpr int NW = (int)(G / 32);                    // words of bits per group
    __shared__ uint32_t wb[8][NW], wt[8][NW];
    __shared__ uint32_t wh[8][128];                      // 2 lmax <= 128 counters per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t w = (uint64_t)blockIdx.x * 8 + warp;
    if (w >= num) return;
    const uint64_t j = order ? order[w] : w;
    const uint64_t i = first + j;
    const DevInst P = inst[i];
    const ExpProg &pg = prog[i];
    const ExpProg8 &pg8 = prog8[i];
    uint4 *etb = g_etb + warp * kProg8MaxTable * (NPT / 4) * 32;   // this warp's exponent table
    const uint32_t half = (uint32_t)((P.n - 1) / 2);
    uint32_t M = (uint32_t)st.m[i];
    uint32_t sig = mont32((uint32_t)st.s[i], sk.lane[lane], sk.p, sk.pinv);
    const uint64_t pos_after = st.pos[i] + per_inst;
    uint32_t *B = wb[warp], *T = wt[warp], *h = wh[warp];
    for (int b = lane; b < 2 * lmax; b += 32) h[b] = 0;
    uint32_t cur_bit = 0, cur_len = 0;                   // run open at the group's start (0: none)
    uint32_t x[NPT], sig_last = sig;
    uint64_t g_last = 0;
    for (uint64_t g0 = 0; g0 < per_inst; g0 += G) {
        uint32_t sv[NPT], msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        messages32<NPT>(P, sk, lane, my0, per_inst, M, sig, sv, msg);
        encrypt32_p8<NPT>(P, pg, pg8, msg, x, etb, lane);
        const uint32_t valid = per_inst - g0 < G ? (uint32_t)(per_inst - g0) : (uint32_t)G;
        uint32_t byte = 0;
#pragma unroll
        for (int u = 0; u < NPT; ++u)
            if (my0 + u < per_inst && x[u] > half) byte |= 1u << u;
        uint32_t word = byte << (8 * (lane & 3));
        word |= __shfl_xor_sync(kFullMask, word, 1);
        word |= __shfl_xor_sync(kFullMask, word, 2);
        if ((lane & 3) == 0) B[lane >> 2] = word;
        __syncwarp();
        if (lane < NW) {
            const uint32_t prev = (B[lane] << 1) | (lane ? B[lane - 1] >> 31 : cur_bit);
            uint32_t t = B[lane] ^ prev;
            if (lane == 0 && cur_len == 0) t |= 1u;      // the call's first number starts a run
            T[lane] = t;
        }
        __syncwarp();
        if (lane == 0 && cur_len && (T[0] & 1u))         // the carried run ended before this group
            atomicAdd(&h[cur_bit * lmax + min(cur_len, (uint32_t)lmax) - 1], 1u);
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            const uint32_t k = NPT * lane + u;
            if (k + 1 >= valid || !((T[(k + 1) >> 5] >> ((k + 1) & 31)) & 1u)) continue;
            // a run ends at k: its start is the highest transition at or below k
            int wi = (int)(k >> 5);
            uint32_t m = T[wi] & (((k & 31) == 31) ? 0xffffffffu : ((2u << (k & 31)) - 1u));
            while (!m && wi > 0) m = T[--wi];
            const uint32_t L = m ? k - (32u * wi + 31u - (uint32_t)__clz(m)) + 1u : k + 1u + cur_len;
            const uint32_t bit = (B[k >> 5] >> (k & 31)) & 1u;
            atomicAdd(&h[bit * lmax + min(L, (uint32_t)lmax) - 1], 1u);
        }
        // carry the run open at the group's end (every lane computes the same)
        {
            const uint32_t last = valid - 1;
            int wi = (int)(last >> 5);
            uint32_t m = T[wi] & (((last & 31) == 31) ? 0xffffffffu : ((2u << (last & 31)) - 1u));
            while (!m && wi > 0) m = T[--wi];
            const uint32_t new_bit = (B[last >> 5] >> (last & 31)) & 1u;
            cur_len = m ? last - (32u * wi + 31u - (uint32_t)__clz(m)) + 1u : cur_len + valid;
            cur_bit = new_bit;
        }
        __syncwarp();
    }
    __syncwarp();
    for (int b = lane; b < 2 * lmax; b += 32)
        if (h[b]) atomicAdd(hist + b, (unsigned long long)h[b]);
    write_state_after<NPT, uint32_t, uint32_t>(st, sk, i, lane, g_last, per_inst, pos_after, M, sig_last,
                                               x);
}

// Collision test (Tests section): each stream's numbers of the call in
// consecutive segments of S (a multiple of the 256-number warp group); the
// count of a segment is the number of its numbers whose bin floor(B R) an
// earlier number of the segment already took, i.e. S minus its distinct bins,
// whatever the order in which they are seen.  Two kernels:
//   coll_bins_kernel: Eq. 9 for `len` numbers of the streams of launch slots
//     [w0, wend), each number's bin written as a 32-bit word in stream order,
//     bins[(w - w0) len + k] (or nothing when store is 0: the numbers past the
//     last complete segment, generated only to advance the streams);
//   coll_count_kernel: one block per segment at a time (persistent), its B
//     bits in shared memory: cleared, every bin set with a shared atomic OR
//     that counts the bits already set, then hist[min(C, H-1)] += 1.
// A B-bit bitmap per segment in shared memory (128 KiB at B = 2^20) replaces
// one bitmap per resident warp in global memory, whose working set (one per
// warp of the GPU) exceeds L2 and makes every OR a DRAM read-modify-write.
template <int NPT>
__global__ void __launch_bounds__(kSerialWarps * 32, PH_SERIAL_MINB)
coll_bins_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog,
                 const ExpProg8 *__restrict__ prog8, DevState st,
                 SkipConst sk, uint64_t first, uint64_t w0, uint64_t wend, uint64_t len, int store,
                 uint32_t B, uint32_t *__restrict__ bins, const uint32_t *__restrict__ order)
{
    constexpr int WB = kSerialWarps;
    constexpr uint64_t G = 32 * NPT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t w = w0 + (uint64_t)blockIdx.x * WB + warp;
    if (w >= wend) return;
    const uint64_t j = order ? order[w] : w;
    const uint64_t i = first + j;
    const DevInst P = inst[i];
    const ExpProg &pg = prog[i];
    const ExpProg8 &pg8 = prog8[i];
    uint4 *etb = g_etb + warp * kProg8MaxTable * (NPT / 4) * 32;   // this warp's exponent table
    const uint32_t r = (uint32_t)(((uint64_t)B << 32) / P.yN);
    uint32_t M = (uint32_t)st.m[i];
    uint32_t sig = mont32((uint32_t)st.s[i], sk.lane[lane], sk.p, sk.pinv);
    const uint64_t pos_after = st.pos[i] + len;
    uint32_t *row = bins + (w - w0) * len;
    uint32_t x[NPT], sig_last = sig;
    uint64_t g_last = 0;
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        uint32_t sv[NPT], msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        const bool full = g0 + G <= len;                 // warp-uniform
        if (full)
            messages32<NPT, true>(P, sk, lane, my0, len, M, sig, sv, msg);
        else
            messages32<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
        encrypt32_p8<NPT>(P, pg, pg8, msg, x, etb, lane);
        if (!store) continue;                            // (len is then the call's tail)
        uint32_t b[NPT];
        serial_bins<NPT>(x, P.yN, P.ybits, r, B, b);
        // stored lengths are whole segments, so every group is full
#pragma unroll
        for (int u = 0; u < NPT; u += 4)
            *reinterpret_cast<uint4 *>(row + my0 + u) = make_uint4(b[u], b[u + 1], b[u + 2], b[u + 3]);
    }
    write_state_after<NPT, uint32_t, uint32_t>(st, sk, i, lane, g_last, len, pos_after, M, sig_last, x);
}

static constexpr int kCollCountThreads = 1024;

// Each thread takes its bins eight at a time; the loads of the next eight
// (of this segment or of the block's next one) are issued before the ORs of
// the current eight, so the reads of one segment overlap the counting, the
// reduction and the bitmap clearing of the previous one.
__device__ __forceinline__ void coll_load8(const uint32_t *__restrict__ bins, uint64_t nseg, uint32_t S,
                                           uint64_t g, uint32_t j, int t, uint32_t (&b)[8])
{
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const uint32_t k = j * 8 * kCollCountThreads + v * kCollCountThreads + t;
        b[v] = g < nseg && k < S ? __ldcs(bins + g * S + k) : 0xFFFFFFFFu;   // bins are below 2^20
    }
}

__global__ void __launch_bounds__(kCollCountThreads)
coll_count_kernel(const uint32_t *__restrict__ bins, uint64_t nseg, uint32_t S, uint32_t B, uint32_t H,
                  unsigned long long *__restrict__ hist)
{
    extern __shared__ uint32_t bm[];                     // ceil(B/32) words
    __shared__ uint32_t part[kCollCountThreads / 32];
    const uint32_t words = (B + 31) / 32;
    const uint32_t nb = (S + 8 * kCollCountThreads - 1) / (8 * kCollCountThreads);   // batches per segment
    const int t = threadIdx.x;
    uint32_t cur[8];
    coll_load8(bins, nseg, S, blockIdx.x, 0, t, cur);
    for (uint64_t g = blockIdx.x; g < nseg; g += gridDim.x) {
        for (uint32_t k = t; k < words; k += kCollCountThreads) bm[k] = 0u;
        __syncthreads();
        uint32_t C = 0;
        for (uint32_t j = 0; j < nb; ++j) {
            uint32_t nxt[8];
            if (j + 1 < nb)
                coll_load8(bins, nseg, S, g, j + 1, t, nxt);
            else
                coll_load8(bins, nseg, S, g + gridDim.x, 0, t, nxt);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if (cur[v] == 0xFFFFFFFFu) continue;
                const uint32_t bit = 1u << (cur[v] & 31);
                C += (atomicOr(bm + (cur[v] >> 5), bit) & bit) ? 1u : 0u;
            }
#pragma unroll
            for (int v = 0; v < 8; ++v) cur[v] = nxt[v];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) C += __shfl_xor_sync(kFullMask, C, off);
        if ((t & 31) == 0) part[t >> 5] = C;
        __syncthreads();
        if (t < 32) {
            C = part[t];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) C += __shfl_xor_sync(kFullMask, C, off);
            if (t == 0) atomicAdd(hist + (C < H ? C : H - 1), 1ull);
        }
        __syncthreads();                                 // bm and part are reused
    }
}

int launch_collision(const GenArgs &a, uint32_t S, uint32_t B, uint32_t H, unsigned long long *hist,
                     uint32_t *bins, uint64_t cap, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t counted = a.per_inst / S * S;        // numbers in complete segments
    const size_t smem = (size_t)((B + 31) / 32) * sizeof(uint32_t);
    int dev = 0, sms = 1, per_sm = 0;
    cudaGetDevice(&dev);
    if (smem > 48 * 1024)                              // above the default 48 KiB (current device)
        cudaFuncSetAttribute(coll_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coll_count_kernel, kCollCountThreads, smem);
    const uint64_t count_blocks = (uint64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    const size_t esm = etb_smem(coll_bins_kernel<8>, kSerialWarps);
    // slots per chunk and numbers per piece so that one piece of one chunk
    // fits the `cap` bins of scratch (at least one segment per slot)
    const uint64_t cw = counted == 0 ? a.num : std::min<uint64_t>(a.num, std::max<uint64_t>(1, cap / S));
    const uint64_t Lp = counted == 0 ? 0 : std::min<uint64_t>(counted, std::max<uint64_t>(S, cap / cw / S * S));
    auto check = [&](const char *what) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) *err = std::string(what) + " launch: " + cudaGetErrorString(e);
        return e == cudaSuccess ? PHPRNG_OK : PHPRNG_ECUDA;
    };
    for (uint64_t w0 = 0; w0 < a.num; w0 += cw) {
        const uint64_t wend = std::min(a.num, w0 + cw);
        const unsigned blocks = (unsigned)((wend - w0 + kSerialWarps - 1) / kSerialWarps);
        for (uint64_t p0 = 0; p0 < counted; p0 += Lp) {
            const uint64_t L = std::min(Lp, counted - p0);
            coll_bins_kernel<8><<<blocks, kSerialWarps * 32, esm, s>>>(a.inst, a.prog, a.prog8, a.st, a.sk, a.first,
                                                                      w0, wend, L, 1, B, bins, a.order);
            int rc = check("coll_bins_kernel");
            if (rc != PHPRNG_OK) return rc;
            const uint64_t nseg = (wend - w0) * (L / S);
            coll_count_kernel<<<(unsigned)std::min(nseg, count_blocks), kCollCountThreads, smem, s>>>(
                bins, nseg, S, B, H, hist);
            rc = check("coll_count_kernel");
            if (rc != PHPRNG_OK) return rc;
        }
        if (a.per_inst > counted) {
            coll_bins_kernel<8><<<blocks, kSerialWarps * 32, esm, s>>>(a.inst, a.prog, a.prog8, a.st, a.sk, a.first,
                                                                      w0, wend, a.per_inst - counted, 0, B, bins,
                                                                      a.order);
            const int rc = check("coll_bins_kernel");
            if (rc != PHPRNG_OK) return rc;
        }
    }
    return PHPRNG_OK;
}

int launch_runs(const GenArgs &a, int lmax, unsigned long long *hist, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    const uint64_t blocks = (a.num + 7) / 8;
    runs_kernel<8><<<(unsigned)blocks, 256, etb_smem(runs_kernel<8>, 8), (cudaStream_t)stream>>>(
        a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, lmax, hist, a.order);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("runs_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}


// Interstream serial test, step 1: bins floor(B R) of a chunk of c (Np
// streams x L numbers, instance-major; uint64 elements when c64, as a
// mixed-width context writes them) written in the paper's interleaved
// order, binsT[j Np + a] for stream a, number j.  A block takes a tile of 32
// streams x 32 numbers through shared memory so that the reads run along a
// stream and the writes along the streams.
// Per-stream bin constants of a call, once: {yN, ybits, floor(B 2^32 / yN)}.
__global__ void __launch_bounds__(256)
inter_consts_kernel(const DevInst *__restrict__ inst, uint64_t first, uint64_t Np, uint32_t B,
                    uint4 *__restrict__ k)
{
    const uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= Np) return;
    const DevInst P = inst[first + a];
    k[a] = make_uint4(P.yN, P.ybits, (uint32_t)(((uint64_t)B << 32) / P.yN), 0u);
}

template <typename BT>
__global__ void __launch_bounds__(256)
inter_bins_kernel(const uint4 *__restrict__ kc, uint64_t Np, uint64_t L, const void *__restrict__ c,
                  int c64, uint32_t B, BT *__restrict__ binsT)
{
    __shared__ uint32_t tile[32][33];
    const uint32_t tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const uint64_t a0 = (uint64_t)blockIdx.x * 32, j0 = (uint64_t)blockIdx.y * 32;
    for (uint32_t r = ty; r < 32; r += 8) {
        const uint64_t a = a0 + r, j = j0 + tx;
        if (a < Np && j < L) {
            const uint4 k = kc[a];
            const uint32_t cv = c64 ? (uint32_t)static_cast<const uint64_t *>(c)[a * L + j]
                                    : static_cast<const uint32_t *>(c)[a * L + j];
            tile[r][tx] = serial_bin(cv, k.x, k.y, k.z, B);
        }
    }
    __syncthreads();
    for (uint32_t r = ty; r < 32; r += 8) {
        const uint64_t j = j0 + r, a = a0 + tx;
        if (j < L && a < Np) binsT[j * Np + a] = (BT)tile[tx][r];
    }
}

// Step 2: consecutive non-overlapping D-tuples of the interleaved bins, one
// count each (per-block shared counters when B^D is at most kInterSmemBins).
// Bins are 16-bit words when B <= 2^16 (half the bytes of both passes).
static constexpr uint32_t kInterSmemBins = 8192;

template <bool SMEM, typename BT>
__global__ void __launch_bounds__(256)
inter_hist_kernel(const BT *__restrict__ binsT, uint64_t ntup, int D, uint32_t B, uint32_t nbins,
                  unsigned long long *__restrict__ hist)
{
    __shared__ uint32_t sh[SMEM ? kInterSmemBins : 1];
    if (SMEM) {
        for (uint32_t b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
        __syncthreads();
    }
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntup;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t idx = 0, scale = 1;
        for (int d = 0; d < D; ++d) {
            idx += (uint32_t)binsT[t * (uint64_t)D + (uint64_t)d] * scale;
            scale *= B;
        }
        if (SMEM) atomicAdd(sh + idx, 1u);
        else atomicAdd(hist + idx, 1ull);
    }
    if (SMEM) {
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nbins; b += blockDim.x)
            if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
    }
}

// Interstream serial test for 2 <= D <= 8, fused: with D dividing the number
// of streams, the interleaved sequence's D-tuples are (number j of streams
// Dq, ..., Dq + D-1), so the D streams of a tuple group run as adjacent warps
// of one block (floor(8/D) groups per block) and meet once per warp group: every warp but the group's first
// leaves its group's bins in shared memory (double-buffered), the D warps pass
// a named barrier of their own (D*32 threads; the groups of a block never wait
// on one another), and the first warp counts the group's tuples.  No bins go
// to HBM and no second kernel runs.  A group waits at most for its slowest
// stream; groups run heaviest first (group_order).  All D warps of a group run
// the same number of warp groups and leave together, so every barrier is
// reached by all of them.
template <int NPT, int GD>
__global__ void __launch_bounds__(GD * (kSerialWarps / GD) * 32, PH_SERIAL_MINB)
inter_groups_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog,
                    const ExpProg8 *__restrict__ prog8, DevState st,
                    SkipConst sk, uint64_t first, uint64_t num, uint64_t len, uint32_t B,
                    unsigned long long *__restrict__ hist, const uint32_t *__restrict__ group_order)
{
    constexpr int NG = kSerialWarps / GD;             // tuple groups per block
    constexpr int WB = GD * NG;                        // warps per block (6 for D = 3, 5 for D = 5, ...)
    static_assert(GD >= 2 && GD <= kSerialWarps && NPT == 8, "groups of warps, 8 bins per lane as one 16-byte row");
    constexpr uint64_t G = 32 * NPT;
    __shared__ uint4 pb[NG][GD - 1][2][32];            // per group: its other streams' bins, two buffers
    __shared__ uint32_t lc[WB][kLocalBins];            // per warp: shared counters when B^D <= kLocalBins
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = warp / GD, member = warp % GD;
    const uint64_t gs = (uint64_t)blockIdx.x * NG + gi;   // group slot
    if ((uint64_t)GD * gs >= num) return;              // num is a multiple of GD: the group leaves together
    const uint64_t gq = group_order ? group_order[gs] : gs;
    const uint64_t j = (uint64_t)GD * gq + member;
    const uint64_t i = first + j;
    const DevInst P = inst[i];
    const ExpProg &pg = prog[i];
    const ExpProg8 &pg8 = prog8[i];
    uint4 *etb = g_etb + warp * kProg8MaxTable * (NPT / 4) * 32;   // this warp's exponent table
    const uint32_t r = (uint32_t)(((uint64_t)B << 32) / P.yN);
    uint32_t nbins = 1;
    for (int d = 0; d < GD && nbins <= kLocalBins; ++d) nbins *= B;
    const bool local = nbins <= kLocalBins;
    uint32_t *cnt = lc[warp];
    if (local)
        for (uint32_t b = lane; b < kLocalBins; b += 32) cnt[b] = 0;
    uint32_t M = (uint32_t)st.m[i];
    uint32_t sig = mont32((uint32_t)st.s[i], sk.lane[lane], sk.p, sk.pinv);
    const uint64_t pos_after = st.pos[i] + len;
    const uint32_t bar = 1 + (uint32_t)gi;             // the group's named barrier (0 is __syncthreads)
    uint32_t x[NPT], sig_last = sig;
    uint64_t g_last = 0;
    int buf = 0;
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        uint32_t sv[NPT], msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        const bool full = g0 + G <= len;               // group-uniform
        if (full)
            messages32<NPT, true>(P, sk, lane, my0, len, M, sig, sv, msg);
        else
            messages32<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
        encrypt32_p8<NPT>(P, pg, pg8, msg, x, etb, lane);
        uint32_t b[NPT];
        serial_bins<NPT>(x, P.yN, P.ybits, r, B, b);
        if (member)
            pb[gi][member - 1][buf][lane] =
                make_uint4(b[0] | b[1] << 16, b[2] | b[3] << 16, b[4] | b[5] << 16, b[6] | b[7] << 16);
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(GD * 32) : "memory");
        if (!member) {
            uint32_t idx[NPT], scale = 1;
#pragma unroll
            for (int u = 0; u < NPT; ++u) idx[u] = b[u];
#pragma unroll
            for (int d = 1; d < GD; ++d) {
                scale *= B;
                const uint4 q = pb[gi][d - 1][buf][lane];
                const uint32_t o[NPT] = {q.x & 0xFFFFu, q.x >> 16, q.y & 0xFFFFu, q.y >> 16,
                                         q.z & 0xFFFFu, q.z >> 16, q.w & 0xFFFFu, q.w >> 16};
#pragma unroll
                for (int u = 0; u < NPT; ++u) idx[u] += o[u] * scale;   // the tuple's first element least significant
            }
#pragma unroll
            for (int u = 0; u < NPT; ++u) {
                if (!full && my0 + u >= len) continue;
                if (local)
                    atomicAdd(cnt + idx[u], 1u);
                else
                    atomicAdd(hist + idx[u], 1ull);
            }
            if (local && (g0 / G) % kLocalFlushGroups == kLocalFlushGroups - 1)
                flush_local<false>(cnt, nbins, lane, hist);
        }
        buf ^= 1;
    }
    if (local && !member) flush_local<false>(cnt, nbins, lane, hist);
    write_state_after<NPT, uint32_t, uint32_t>(st, sk, i, lane, g_last, len, pos_after, M, sig_last, x);
}

template <int GD>
static void launch_groups_d(const GenArgs &a, uint32_t B, unsigned long long *hist, const uint32_t *group_order,
                            cudaStream_t s)
{
    constexpr int WB = GD * (kSerialWarps / GD);
    const uint64_t blocks = (a.num + WB - 1) / WB;
    inter_groups_kernel<8, GD><<<(unsigned)blocks, WB * 32, etb_smem(inter_groups_kernel<8, GD>, WB), s>>>(
        a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, B, hist, group_order);
}

int launch_inter_groups(const GenArgs &a, int D, uint32_t B, unsigned long long *hist,
                        const uint32_t *group_order, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    switch (D) {
    case 2: launch_groups_d<2>(a, B, hist, group_order, s); break;
    case 3: launch_groups_d<3>(a, B, hist, group_order, s); break;
    case 4: launch_groups_d<4>(a, B, hist, group_order, s); break;
    case 5: launch_groups_d<5>(a, B, hist, group_order, s); break;
    case 6: launch_groups_d<6>(a, B, hist, group_order, s); break;
    case 7: launch_groups_d<7>(a, B, hist, group_order, s); break;
    case 8: launch_groups_d<8>(a, B, hist, group_order, s); break;
    default:
        *err = "inter_groups_kernel: D must be 2 to 8";
        return PHPRNG_EINVAL;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("inter_groups_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_inter_consts(const DevInst *inst, uint64_t first, uint64_t Np, uint32_t B, void *k, void *stream,
                        std::string *err)
{
    if (Np == 0) return PHPRNG_OK;
    inter_consts_kernel<<<(unsigned)((Np + 255) / 256), 256, 0, (cudaStream_t)stream>>>(inst, first, Np, B,
                                                                                          (uint4 *)k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("inter_consts_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_interstream(const void *k, uint64_t Np, uint64_t L, const void *c, int c64,
                       int D, uint32_t B, uint32_t *binsT, unsigned long long *hist, void *stream,
                       std::string *err)
{
    if (Np == 0 || L == 0) return PHPRNG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (L > kInterMaxChunk) {                      // grid.y limit: 65,535 tiles of 32
        *err = "interstream chunk longer than 65,535 x 32 numbers";
        return PHPRNG_EINVAL;
    }
    const dim3 grid((unsigned)((Np + 31) / 32), (unsigned)((L + 31) / 32));
    const bool narrow = B <= 65536u;                 // bins fit 16 bits
    uint16_t *bins16 = reinterpret_cast<uint16_t *>(binsT);
    if (narrow)
        inter_bins_kernel<uint16_t><<<grid, 256, 0, s>>>((const uint4 *)k, Np, L, c, c64, B, bins16);
    else
        inter_bins_kernel<uint32_t><<<grid, 256, 0, s>>>((const uint4 *)k, Np, L, c, c64, B, binsT);
    uint32_t nbins = 1;
    for (int d = 0; d < D; ++d) nbins *= B;
    const uint64_t ntup = Np * L / (uint64_t)D;
    if (ntup) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t want = (ntup + 255) / 256, cap = (uint64_t)sms * 8;
        const unsigned blocks = (unsigned)(want < cap ? want : cap);
        if (narrow) {
            if (nbins <= kInterSmemBins)
                inter_hist_kernel<true, uint16_t><<<blocks, 256, 0, s>>>(bins16, ntup, D, B, nbins, hist);
            else
                inter_hist_kernel<false, uint16_t><<<blocks, 256, 0, s>>>(bins16, ntup, D, B, nbins, hist);
        } else {
            if (nbins <= kInterSmemBins)
                inter_hist_kernel<true, uint32_t><<<blocks, 256, 0, s>>>(binsT, ntup, D, B, nbins, hist);
            else
                inter_hist_kernel<false, uint32_t><<<blocks, 256, 0, s>>>(binsT, ntup, D, B, nbins, hist);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("interstream kernels: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_serial(const GenArgs &a, int D, uint32_t B, unsigned long long *hist, void *stream,
                  std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    const uint64_t blocks = (a.num + kSerialWarps - 1) / kSerialWarps;
    if (D == 0)                                      // the poker test
        serial_kernel<8, true, kSerialWarps><<<(unsigned)blocks, kSerialWarps * 32,
                                               etb_smem(serial_kernel<8, true, kSerialWarps>, kSerialWarps),
                                               (cudaStream_t)stream>>>(
            a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, 5, 10, hist, a.order);
    else
        serial_kernel<8, false, kSerialWarps><<<(unsigned)blocks, kSerialWarps * 32,
                                                etb_smem(serial_kernel<8, false, kSerialWarps>, kSerialWarps),
                                                (cudaStream_t)stream>>>(
            a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, D, B, hist, a.order);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("serial_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

}  // namespace phprng
