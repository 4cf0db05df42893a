// skipdev.cuh -- device side of the closed-form skip-ahead (Eq. 7).
//
// With s = a^L mod p (L the cycle position of s, a a primitive root), a skip
// of k = q(p-1) + r steps gives (Eq. 7)
//     s' = s a^r mod p = a^((L + r) mod (p-1)),
//     m' = m + q p(p-1)/2 + sum_{j=1..r} (a^(L+j) mod p)   (mod n),
// and the sum is Pref(L + r) - Pref(L), wrapping once around the cycle
// (Pref(p-1) = p(p-1)/2) when L + r > p-1.  Pref(t) is read from the exact
// prefix table at the checkpoint floor(t/B)*B plus a tail of fewer than B
// terms that the 32 lanes of a warp share (B/32 each), starting from the
// checkpoint power P[j] times the lane constant a^(32 l).
#pragma once
#include "arith.cuh"
#include "internal.h"

namespace phprng {

// Pref(t) and a^t mod p for 0 <= t <= p-1; every lane of the warp calls it and
// every lane gets both results.
__device__ __forceinline__ void pref_warp(const SkipTable &tb, uint64_t t, uint64_t *sum_out,
                                          uint32_t *pow_out)
{
    const int lane = threadIdx.x & 31;
    const uint64_t j = t >> kSkipLog2B;
    const uint32_t cnt = (uint32_t)(t - (j << kSkipLog2B));       // terms after the checkpoint
    const uint32_t Pj = tb.P[j];
    uint32_t x = mont32(Pj, tb.laneM[lane], tb.p, tb.pinv);        // a^(jB + 32 lane)
    const uint32_t lo = 32u * (uint32_t)lane;
    uint64_t sum = 0;
    uint32_t last = x;
#pragma unroll 8
    for (uint32_t u = 1; u <= kSkipB / 32; ++u) {
        x = mont32(x, tb.aM, tb.p, tb.pinv);                       // a^(jB + lo + u)
        if (lo + u <= cnt) {
            sum += x;
            last = x;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    const uint32_t owner = cnt ? (cnt - 1) >> 5 : 0;
    const uint32_t pw = __shfl_sync(0xffffffffu, last, owner);
    *sum_out = tb.T[j] + sum;
    *pow_out = cnt ? pw : Pj;
}

// sum_{j=1..r} (a^(L+j) mod p) and a^((L+r) mod (p-1)), for L, r in [0, p-2].
__device__ __forceinline__ void window_warp(const SkipTable &tb, uint64_t L, uint64_t r,
                                            uint64_t *sum_out, uint32_t *pow_out)
{
    const uint64_t pm1 = tb.p - 1;
    uint64_t s0, s1;
    uint32_t w0, w1;
    pref_warp(tb, L, &s0, &w0);
    if (r == 0) {
        *sum_out = 0;
        *pow_out = w0;
        return;
    }
    const uint64_t hi = L + r;
    if (hi <= pm1) {
        pref_warp(tb, hi, &s1, &w1);
        *sum_out = s1 - s0;
    } else {
        pref_warp(tb, hi - pm1, &s1, &w1);
        *sum_out = (tb.half - s0) + s1;
    }
    *pow_out = w1;
}

// State k steps after (m, s = a^L) by Eq. 7.  The message update is exact:
// q mod n times p(p-1)/2 mod n, plus the window sum mod n, all mod n.
// For the constant skip (kind 1) L carries b = s0: m' = m + k b mod n, s' = b
// (Eq. 3 with s_k = b: the k messages after m are m + b, m + 2b, ...).
__device__ __forceinline__ void skip_state_warp(const SkipTable &tb, const DevInst &P,
                                                uint64_t m, uint64_t L, uint64_t k,
                                                uint64_t *m_out, uint32_t *s_out,
                                                uint64_t *L_out)
{
    if (tb.kind == 1) {
        const uint64_t n = P.n, b = L;
        uint64_t add;
        if (!P.wide) {
            add = ((k % n) * b) % n;                               // b < 2^32 > n: fits 64 bits
            *m_out = (m + add) % n;
        } else {
            const uint64_t t = mont64(k % n, b % n, n, P.ninv);     // k b R^-1
            add = mont64(t, P.aux, n, P.ninv);                     // k b mod n
            *m_out = addmod64(m, add, n);
        }
        *s_out = (uint32_t)b;
        *L_out = b;
        return;
    }
    const uint64_t pm1 = tb.p - 1;
    const uint64_t q = k / pm1, r = k - q * pm1;
    uint64_t W;
    uint32_t s;
    window_warp(tb, L, r, &W, &s);
    const uint64_t n = P.n;
    uint64_t add;
    if (!P.wide) {
        add = ((q % n) * (tb.half % n)) % n;
        add = (add + W % n) % n;
        *m_out = (m + add) % n;
    } else {
        const uint64_t t = mont64(q % n, tb.half % n, n, P.ninv);   // q*half*R^-1
        add = mont64(t, P.aux, n, P.ninv);                         // q*half mod n
        add = addmod64(add, W % n, n);
        *m_out = addmod64(m, add, n);
    }
    *s_out = s;
    *L_out = (L + r) % pm1;
}

}  // namespace phprng
