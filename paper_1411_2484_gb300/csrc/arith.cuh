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

// hi - u, plus n when that borrows: the last step of the subtractive
// Montgomery reduction (hi, u < n).
#ifndef PH_FINISH
#define PH_FINISH 0
#endif
PH_HD uint32_t mont_finish32(uint32_t hi, uint32_t u, uint32_t n)
{
#if PH_FINISH == 1
    return hi - u + (hi < u ? n : 0u);
#elif PH_FINISH == 2 && defined(__CUDA_ARCH__)
    uint32_t r;
    asm("{\n\t.reg .u32 t, m;\n\t"
        "sub.cc.u32 t, %1, %2;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "and.b32 m, m, %3;\n\t"
        "add.u32 %0, t, m;\n\t}"
        : "=r"(r) : "r"(hi), "r"(u), "r"(n));
    return r;
#else
    const uint32_t t = hi - u;
    return hi < u ? t + n : t;
#endif
}

PH_HD uint32_t mont32(uint32_t a, uint32_t b, uint32_t n, uint32_t ninv)
{
    uint64_t T = (uint64_t)a * b;
    uint32_t lo = (uint32_t)T, hi = (uint32_t)(T >> 32);
    uint32_t q = lo * ninv;
    uint32_t u = umulhi32(q, n);
    return mont_finish32(hi, u, n);
}

// Montgomery product by a constant b with bq = b n^-1 mod 2^32 precomputed:
// the low word of a b is needed only to form q = lo(a b) n^-1 = a bq mod 2^32,
// and the subtractive form never reads it otherwise (lo(q n) = lo(a b)), so
// three multiplies replace four.
PH_HD uint32_t mont32c(uint32_t a, uint32_t b, uint32_t bq, uint32_t n)
{
    const uint32_t hi = umulhi32(a, b);
    const uint32_t q = a * bq;
    const uint32_t u = umulhi32(q, n);
    return mont_finish32(hi, u, n);
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

// a + b reduced only when it wraps past 2^32, for any a < 2^32 and b < n: the
// result is below 2^32 and congruent to a + b mod n (a wrapped sum exceeds n,
// and a + b - n < 2^32 because b < n), not necessarily below n.
PH_HD uint32_t addmod32_lazy(uint32_t a, uint32_t b, uint32_t n)
{
#if defined(__CUDA_ARCH__)
    // both sums as separate PTX additions (a + b and (a + b) - n), chosen by
    // the carry of the first: measured one instruction shorter than the
    // conditional subtraction written in C
    uint32_t t, r;
    asm("add.u32 %0, %1, %2;" : "=r"(t) : "r"(a), "r"(b));
    asm("sub.u32 %0, %1, %2;" : "=r"(r) : "r"(t), "r"(n));
    return t < b ? r : t;
#else
    const uint32_t t = a + b;
    return t < b ? t - n : t;
#endif
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

// Exponentiation program: the left-to-right sliding-window decomposition of
// one instance's exponent (Menezes, van Oorschot, Vanstone, Handbook of
// Applied Cryptography, Algorithm 14.85), built on the host.  The table holds
// the odd powers m, m^3, .., m^(2 tbl - 1); x starts as the table entry of the
// first window, then each later window is `sq` squarings followed by one
// product with its table entry, then `tail` squarings close the exponent.
// One byte per window: sq in bits 0-5, table index in bits 6-7.
struct alignas(16) ExpProg {
    uint8_t nent;       // windows (>= 1)
    uint8_t tail;       // squarings after the last window
    uint8_t tbl;        // table entries: 1, 2 or 4
    uint8_t pad;
    uint8_t ent[28];
};

// Exponent program of the 32-bit kernels: a table of 1 to kProg8MaxTable odd
// powers m, m^3, .., m^(2 tbl - 1) (shared memory holds it), the table size
// and the windows chosen per exponent by an exact search (dynamic programming
// over the exponent's bit positions, for every table size) for the fewest
// Montgomery products, table included.  x starts as the first window's table
// entry; each later window is `sq` squarings then one product with its entry
// (e is odd, so no squarings follow the last window).  K, Kq: this program's
// exit constant R^(1-alpha) mod n and K n^-1 mod 2^32.
struct alignas(16) ExpProg8 {
    uint32_t K, Kq;
    uint8_t nent;       // windows (>= 1)
    uint8_t tbl;        // table entries, 1 .. kProg8MaxTable
    uint8_t pad[2];
    uint16_t ent[32];   // per window: sq in bits 0-7, table index (v-1)/2 in bits 8-10
};
static_assert(sizeof(ExpProg8) == 80, "ExpProg8 layout");
// Largest table the host search allows: 6 rows of a warp's 8 numbers per lane
// are 6 KiB of shared memory (the entry field could index 8).  Over random
// 32-bit exponents a cap of 6 costs 0.04 products per exponentiation against 8.
static constexpr int kProg8MaxTable = 6;

// The same program run with the table in an array (host tests, NPT numbers).
template <int NPT>
PH_HD void modexp_prog8(uint32_t (&x)[NPT], const uint32_t (&m)[NPT], const ExpProg8 &pg, uint32_t n,
                        uint32_t ninv)
{
    uint32_t t[8][NPT], m2[NPT];
    for (int u = 0; u < NPT; ++u) t[0][u] = m[u];
    if (pg.tbl >= 2)
        for (int u = 0; u < NPT; ++u) m2[u] = mont32(m[u], m[u], n, ninv);
    for (int k = 1; k < pg.tbl; ++k)
        for (int u = 0; u < NPT; ++u) t[k][u] = mont32(t[k - 1][u], m2[u], n, ninv);
    for (int u = 0; u < NPT; ++u) x[u] = t[pg.ent[0] >> 8][u];
    for (int k = 1; k < pg.nent; ++k) {
        for (int q = 0; q < (pg.ent[k] & 0xFF); ++q)
            for (int u = 0; u < NPT; ++u) x[u] = mont32(x[u], x[u], n, ninv);
        for (int u = 0; u < NPT; ++u) x[u] = mont32(x[u], t[(pg.ent[k] >> 8) & 7][u], n, ninv);
    }
    for (int u = 0; u < NPT; ++u) x[u] = mont32c(x[u], pg.K, pg.Kq, n);
}

PH_HD uint32_t mont(uint32_t a, uint32_t b, uint32_t n, uint32_t ninv) { return mont32(a, b, n, ninv); }
PH_HD uint64_t mont(uint64_t a, uint64_t b, uint64_t n, uint64_t ninv) { return mont64(a, b, n, ninv); }
// The exit product x K of an exponentiation (Kq = K n^-1 mod 2^32 on the 32-bit path).
PH_HD uint32_t mont_exit(uint32_t x, uint32_t K, uint32_t Kq, uint32_t n, uint32_t) { return mont32c(x, K, Kq, n); }
PH_HD uint64_t mont_exit(uint64_t x, uint64_t K, uint64_t, uint64_t n, uint64_t ninv) { return mont64(x, K, n, ninv); }

// x_u = MP(x_u, y_u) for every u.  The 32-bit form is written phase by phase
// across the NPT independent products (all full products, then all q, then
// all high halves, then the corrections), so that consecutive multiplies never
// wait on each other.
template <int NPT>
PH_HD void mont32_vec(uint32_t (&x)[NPT], const uint32_t (&y)[NPT], uint32_t n, uint32_t ninv)
{
    uint32_t lo[NPT], hi[NPT];
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        const uint64_t T = (uint64_t)x[u] * y[u];
        lo[u] = (uint32_t)T;
        hi[u] = (uint32_t)(T >> 32);
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) lo[u] *= ninv;                 // q
#pragma unroll
    for (int u = 0; u < NPT; ++u) lo[u] = umulhi32(lo[u], n);    // hi(q n)
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont_finish32(hi[u], lo[u], n);
}

template <int NPT, typename W>
PH_HD void mont_vec(W (&x)[NPT], const W (&y)[NPT], W n, W ninv)
{
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont(x[u], y[u], n, ninv);
}

template <int NPT>
PH_HD void mont_vec(uint32_t (&x)[NPT], const uint32_t (&y)[NPT], uint32_t n, uint32_t ninv)
{
    mont32_vec<NPT>(x, y, n, ninv);
}

template <int NPT, typename W>
PH_HD void mont_sqr_vec(W (&x)[NPT], W n, W ninv)
{
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont(x[u], x[u], n, ninv);
}

template <int NPT>
PH_HD void mont_sqr_vec(uint32_t (&x)[NPT], uint32_t n, uint32_t ninv)
{
    mont32_vec<NPT>(x, x, n, ninv);
}

// c_u = m_u^e mod n for NPT messages by the exponent's program (Eq. 9c with
// fewer products than the binary method), closed by one product with the
// exit constant K the host derived for that program (Kq = K n^-1 mod 2^32 for
// the 32-bit path, unused on the 64-bit one).  All control flow
// depends only on the program, so it is uniform across a warp that shares
// the instance.
template <int NPT, typename W>
PH_HD void modexp_prog(W (&x)[NPT], const W (&m)[NPT], const ExpProg &pg, W n, W ninv, W K, W Kq)
{
    W t3[NPT], t5[NPT], t7[NPT];
    const int tbl = pg.tbl;
    if (tbl >= 2) {
        W m2[NPT];
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            m2[u] = mont(m[u], m[u], n, ninv);
            t3[u] = mont(m2[u], m[u], n, ninv);
        }
        if (tbl == 4) {
#pragma unroll
            for (int u = 0; u < NPT; ++u) {
                t5[u] = mont(t3[u], m2[u], n, ninv);
                t7[u] = mont(t5[u], m2[u], n, ninv);
            }
        }
    }
    switch (pg.ent[0] >> 6) {
    case 0:
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = m[u];
        break;
    case 1:
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = t3[u];
        break;
    case 2:
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = t5[u];
        break;
    default:
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = t7[u];
        break;
    }
    const int nent = pg.nent;
    int bnext = pg.ent[1];
    for (int k = 1; k < nent; ++k) {
        const int b = bnext;
        bnext = pg.ent[k + 1 < (int)sizeof pg.ent ? k + 1 : k];   // next entry, loaded early
        int sq = b & 63;
        for (; sq >= 2; sq -= 2) {
            mont_sqr_vec<NPT>(x, n, ninv);
            mont_sqr_vec<NPT>(x, n, ninv);
        }
        if (sq) mont_sqr_vec<NPT>(x, n, ninv);
        switch (b >> 6) {
        case 0: mont_vec<NPT>(x, m, n, ninv); break;
        case 1: mont_vec<NPT>(x, t3, n, ninv); break;
        case 2: mont_vec<NPT>(x, t5, n, ninv); break;
        default: mont_vec<NPT>(x, t7, n, ninv); break;
        }
    }
    for (int sq = pg.tail; sq > 0; --sq) mont_sqr_vec<NPT>(x, n, ninv);
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont_exit(x[u], K, Kq, n, ninv);
}

PH_HD int clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

PH_HD double u64_to_double_rn(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __ull2double_rn(x);
#else
    return (double)x;
#endif
}

// Round-to-nearest-even double of the 128-bit integer hi*2^64 + lo.  The top
// 64 significant bits are converted with one RN conversion after the bits
// shifted out are folded into bit 0 (a sticky bit: the conversion rounds at
// bit 11, so only whether the discarded part is zero matters there); the
// power-of-two scaling is exact.
PH_HD double u128_to_double(uint64_t hi, uint64_t lo)
{
    if (hi == 0) return u64_to_double_rn(lo);
    const int sh = 64 - clz64(hi);                       // 1 .. 64
    const uint64_t top = sh == 64 ? hi : (hi << (64 - sh)) | (lo >> sh);
    const uint64_t rest = sh == 64 ? lo : (lo << (64 - sh));
    const double t = u64_to_double_rn(top | (rest != 0 ? 1u : 0u));
    return t * bits_to_double((uint64_t)(1023 + sh) << 52);
}

// floor(256 R) for a double R in [0, 1] taken apart as integers: R =
// sig 2^(ef-1075) with the implicit bit in sig, so 256 R = sig 2^(ef-1067).
PH_HD uint32_t hist_bin256(double R)
{
    uint64_t b;
#if defined(__CUDA_ARCH__)
    b = (uint64_t)__double_as_longlong(R);
#else
    __builtin_memcpy(&b, &R, 8);
#endif
    const int ef = (int)(b >> 52);
    if (ef == 0) return 0;
    const uint64_t sig = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int shift = 1067 - ef;
    const uint32_t bin = shift >= 64 ? 0u : shift <= 0 ? 256u : (uint32_t)(sig >> shift);
    return bin > 255u ? 255u : bin;
}

// floor(256 (c+1)/(n+1)) from integers, for n < 2^32: with y = n+1
// normalised to yN = y 2^(32-ybits) (top bit set) and vN = (c+1) 2^(32-ybits)
// < yN, the estimate floor(vN r / 2^32) with r = floor(2^40 / yN) is the bin or
// one below it (r is short of 2^40/yN by less than 1, and vN < 2^32), and one
// exact comparison decides.  Equal to hist_bin256 of the correctly rounded R:
// a rounding can only reach a multiple of 1/256 that R equals exactly, since
// a nonzero |k/256 - (c+1)/(n+1)| is at least 2^-40, far above half an ulp.
PH_HD uint32_t hist_bin256_int(uint32_t c, uint32_t yN, uint32_t ybits, uint32_t r)
{
    const uint32_t vN = (c + 1) << (32 - ybits);
    uint32_t est = umulhi32(vN, r);
    if ((uint64_t)(est + 1) * yN <= ((uint64_t)vN << 8)) ++est;
    return est;
}

// Funnel shifts of the 64-bit value hi:lo: the high word of (hi:lo) << s and
// the low word of (hi:lo) >> s, 0 <= s <= 31 (one instruction each on the GPU).
PH_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, s);
#else
    return (uint32_t)(((((uint64_t)hi << 32) | lo) << s) >> 32);
#endif
}

PH_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, s);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> s);
#endif
}

// The same double, deciding the rounding from an 11-bit fraction: with
// W = floor((2^95 - 1) / yN), Xf = floor(A W / 2^(32-extra)) is the exact
// quotient X = A 2^(52+extra) / yN scaled by 2^11 (so Xf < 2^64) and short of
// it by less than 3 units of its last bit, because W is short of 2^95/yN by
// at most 1, A < 2^32, and the floor drops less than 1.  Ties are impossible
// (X is an integer or not dyadic, as yN < 2^32), so X rounds up exactly when
// its fraction exceeds 1/2; the 11-bit fraction f of Xf decides that unless
// 1021 <= f < 1024, where the exact remainder of floor(X) = floor(Xf / 2^11)
// decides it (about 1 number in 700).  Outside that band the rounded
// significand is floor((Xf + 2^10) / 2^11) (Xf + 2^10 < 2^64: X < 2^53 - 2^20).
// The arithmetic is kept in 32-bit words: Xf from the two partial products by
// funnel shifts by `extra`, and the high word of the double as
// ((1022 + E) << 20) + Q_hi with E = 32 - lz - ybits - extra (Q carries the
// implicit bit, which lifts the exponent field by one to 1023 + E).
// real32_est is the branch-free part: the double rounded from the 11-bit
// fraction, with *amb = 1 when f lies in the band; real32_exact forms the same
// Xf and decides by the exact remainder; real32_fast does both in one, with
// a branch on the band.
PH_HD double real32_est(uint32_t c, uint32_t yN, uint32_t ybits, uint64_t W, uint32_t *amb)
{
    const uint32_t x = c + 1;
    const uint32_t lz = (uint32_t)clz32(x);
    const uint32_t A = x << lz;
    const uint32_t extra = A < yN ? 1u : 0u;
    // Xf = floor(A W / 2^(32 - extra)): H = A w1 + floor(A w0 / 2^32) (< 2^64,
    // and < 2^63 when extra = 1, as A/yN < 1 then), shifted left by extra
    // with the next bit of A w0 shifted in.
    const uint64_t P = (uint64_t)A * (uint32_t)W;                        // A * w0
    const uint64_t H = (uint64_t)A * (uint32_t)(W >> 32) + (P >> 32);    // A * w1 + hi
    const uint32_t Hlo = (uint32_t)H, Hhi = (uint32_t)(H >> 32);
    const uint32_t Xhi = funnel_l(Hlo, Hhi, extra), Xlo = funnel_l((uint32_t)P, Hlo, extra);
    *amb = (Xlo & 0x7FFu) - 1021u < 3u ? 1u : 0u;
    const uint64_t Xr = (((uint64_t)Xhi << 32) | Xlo) + 1024u;
    const uint32_t Qlo = funnel_r((uint32_t)Xr, (uint32_t)(Xr >> 32), 11);
    const uint32_t Qhi = (uint32_t)(Xr >> 43);
    const uint32_t hi = ((1054u - ybits - lz - extra) << 20) + Qhi;
    return bits_to_double(((uint64_t)hi << 32) | Qlo);
}

PH_HD double real32_exact(uint32_t c, uint32_t yN, uint32_t ybits, uint64_t W)
{
    const uint32_t x = c + 1;
    const uint32_t lz = (uint32_t)clz32(x);
    const uint32_t A = x << lz;
    const uint32_t extra = A < yN ? 1u : 0u;
    const uint64_t P = (uint64_t)A * (uint32_t)W;
    const uint64_t H = (uint64_t)A * (uint32_t)(W >> 32) + (P >> 32);
    const uint64_t Xf = (H << extra) | (extra ? (uint64_t)((uint32_t)P >> 31) : 0u);
    uint64_t Q = Xf >> 11;
    const uint64_t r = ((uint64_t)A << (52 + extra)) - Q * (uint64_t)yN;   // exact, < yN
    Q += (r << 1) > yN ? 1u : 0u;
    const uint32_t hi = ((1054u - ybits - lz - extra) << 20) + (uint32_t)(Q >> 32);
    return bits_to_double(((uint64_t)hi << 32) | (uint32_t)Q);
}

PH_HD double real32_fast(uint32_t c, uint32_t yN, uint32_t ybits, uint64_t W)
{
    const uint32_t x = c + 1;
    const uint32_t lz = (uint32_t)clz32(x);
    const uint32_t A = x << lz;
    const uint32_t extra = A < yN ? 1u : 0u;
    const uint64_t P = (uint64_t)A * (uint32_t)W;                        // A * w0
    const uint64_t H = (uint64_t)A * (uint32_t)(W >> 32) + (P >> 32);    // A * w1 + hi
    const uint32_t Hlo = (uint32_t)H, Hhi = (uint32_t)(H >> 32);
    const uint32_t Xhi = funnel_l(Hlo, Hhi, extra), Xlo = funnel_l((uint32_t)P, Hlo, extra);
    const uint32_t f = Xlo & 0x7FFu;
    uint32_t Qlo, Qhi;
    if (f - 1021u >= 3u) {
        const uint64_t Xr = (((uint64_t)Xhi << 32) | Xlo) + 1024u;
        Qlo = funnel_r((uint32_t)Xr, (uint32_t)(Xr >> 32), 11);
        Qhi = (uint32_t)(Xr >> 43);
    } else {
        uint64_t Q = (((uint64_t)Xhi << 32) | Xlo) >> 11;
        const uint64_t r = ((uint64_t)A << (52 + extra)) - Q * (uint64_t)yN;   // exact, < yN
        Q += (r << 1) > yN ? 1u : 0u;
        Qlo = (uint32_t)Q;
        Qhi = (uint32_t)(Q >> 32);
    }
    const uint32_t hi = ((1054u - ybits - lz - extra) << 20) + Qhi;
    return bits_to_double(((uint64_t)hi << 32) | Qlo);
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
