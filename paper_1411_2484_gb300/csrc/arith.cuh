// arith.cuh -- modular arithmetic of the generator's hot path.
//
// Compiles as CUDA device code (the kernels) and as plain C++ (a host
// build used by the CPU test of the integer-built R).
//
//  mont32 / mont64   Montgomery product a*b*2^-32 mod n (resp. 2^-64), with
//                    the subtractive reduction: q = lo(a b) * n^-1 mod 2^w makes
//                    a b - q n divisible by 2^w exactly, so the result is
//                    hi(a b) - hi(q n), plus n when that borrows.  Inputs < n,
//                    output in [0, n); no intermediate exceeds 2w bits, so any
//                    odd n < 2^w works.
//  addmod32 / 64     (a + b) mod n for a, b < n (Eq. 9b).
//  real32            R = (c+1)/(n+1) correctly rounded (Eq. 9d), built from
//                    integers: quotient by a fixed-point reciprocal of the
//                    normalised divisor, then an exact remainder correction
//                    (Granlund and Montgomery, "Division by invariant integers
//                    using multiplication", PLDI 1994), then round-to-nearest-
//                    even on the remainder.  Equals the IEEE double division
//                    of the two exact operands.
//  real64            RN(RN(c+1) / RN(n+1)) with the hardware FP64 division.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define PH_HD __host__ __device__ __forceinline__
#else
#define PH_HD inline
#endif

namespace phprng {

PH_HD uint32_t umulhi32(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

PH_HD uint64_t umulhi64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

PH_HD int clz32(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

PH_HD double bits_to_double(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    __builtin_memcpy(&d, &b, 8);
    return d;
#endif
}

PH_HD uint32_t mont32(uint32_t a, uint32_t b, uint32_t n, uint32_t ninv)
{
    uint64_t T = (uint64_t)a * b;
    uint32_t lo = (uint32_t)T, hi = (uint32_t)(T >> 32);
    uint32_t q = lo * ninv;
    uint32_t u = umulhi32(q, n);
    uint32_t t = hi - u;
    return hi < u ? t + n : t;
}

PH_HD uint64_t mont64(uint64_t a, uint64_t b, uint64_t n, uint64_t ninv)
{
    uint64_t lo = a * b, hi = umulhi64(a, b);
    uint64_t q = lo * ninv;
    uint64_t u = umulhi64(q, n);
    uint64_t t = hi - u;
    return hi < u ? t + n : t;
}

PH_HD uint32_t addmod32(uint32_t a, uint32_t b, uint32_t n)
{
    uint32_t t = a + b;                 // wraps when a + b >= 2^32 (then a + b > n)
    return (t < a || t >= n) ? t - n : t;
}

PH_HD uint64_t addmod64(uint64_t a, uint64_t b, uint64_t n)
{
    uint64_t t = a + b;
    return (t < a || t >= n) ? t - n : t;
}

// (a - b) mod n for a, b < n.
PH_HD uint32_t submod32(uint32_t a, uint32_t b, uint32_t n)
{
    return a >= b ? a - b : a - b + n;
}

// Bits of the double RN((c+1)/(n+1)) for c < n < 2^32 from the per-instance
// constants yN = (n+1) << (32 - ybits), ybits = bitlen(n+1),
// V = floor(2^84 / yN).
//
// x = c+1 is normalised to A = x << (32 - bitlen(x)) in [2^31, 2^32); with
// extra = (A < yN) the quotient A 2^extra / yN lies in [1, 2) and
// x/y = (A 2^extra / yN) 2^E with E = bitlen(x) - ybits - extra <= -1.
// The 53-bit significand is Q = floor(A 2^(52+extra) / yN) rounded to
// nearest-even by its remainder r:
//   Q' = floor(A V / 2^(32-extra)) is Q, Q-1 or Q-2 (V is short of 2^84/yN by
//   less than 1 and A < 2^32), so at most two corrections of r = A 2^(52+extra)
//   - Q' yN (exact below 3 yN, hence exact mod 2^64) give Q and r < yN.
// Q < 2^53 - 2^20 because A < 2 yN, so rounding never carries into the
// exponent, and the result is a normal double (E >= -34).
PH_HD double real32(uint32_t c, uint32_t yN, uint32_t ybits, uint64_t V)
{
    uint32_t x = c + 1;
    int xb = 32 - clz32(x);
    uint32_t A = x << (32 - xb);
    uint32_t extra = A < yN ? 1u : 0u;
    int E = xb - (int)ybits - (int)extra;
    uint64_t P = (uint64_t)A * (uint32_t)V;            // A * v0
    uint64_t H = (uint64_t)A * (uint32_t)(V >> 32);    // A * v1
    uint64_t Q = (H << extra) + (P >> (32 - extra));
    uint64_t r = ((uint64_t)A << (52 + extra)) - Q * (uint64_t)yN;
    if (r >= yN) { r -= yN; ++Q; }
    if (r >= yN) { r -= yN; ++Q; }
    uint64_t r2 = r << 1;
    Q += (r2 > yN || (r2 == yN && (Q & 1))) ? 1u : 0u;
    return bits_to_double(((uint64_t)(1022 + E) << 52) + Q);
}

// c_u = msg_u^e mod n for NPT independent messages (Eq. 9c): left-to-right
// square-and-multiply over the ebits bits of e on Montgomery products started
// from the plain messages, then one product with K = R^(1-alpha) mod n (the
// host derives alpha, the net power of R^-1 the products leave behind).  The
// bit test is uniform across a warp that shares e, and the NPT chains are
// independent, which is the instruction-level parallelism of a lane.
template <int NPT>
PH_HD void modexp32(uint32_t (&x)[NPT], const uint32_t (&msg)[NPT], uint32_t e, int ebits,
                    uint32_t n, uint32_t ninv, uint32_t K)
{
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = msg[u];
    for (int b = ebits - 2; b >= 0; --b) {
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = mont32(x[u], x[u], n, ninv);
        if ((e >> b) & 1u) {
#pragma unroll
            for (int u = 0; u < NPT; ++u) x[u] = mont32(x[u], msg[u], n, ninv);
        }
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont32(x[u], K, n, ninv);
}

template <int NPT>
PH_HD void modexp64(uint64_t (&x)[NPT], const uint64_t (&msg)[NPT], uint64_t e, int ebits,
                    uint64_t n, uint64_t ninv, uint64_t K)
{
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = msg[u];
    for (int b = ebits - 2; b >= 0; --b) {
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = mont64(x[u], x[u], n, ninv);
        if ((e >> b) & 1ull) {
#pragma unroll
            for (int u = 0; u < NPT; ++u) x[u] = mont64(x[u], msg[u], n, ninv);
        }
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont64(x[u], K, n, ninv);
}

PH_HD double real64(uint64_t c, uint64_t n)
{
#if defined(__CUDA_ARCH__)
    return __ddiv_rn(__ull2double_rn(c + 1), __ull2double_rn(n + 1));
#else
    return (double)(c + 1) / (double)(n + 1);
#endif
}

}  // namespace phprng
