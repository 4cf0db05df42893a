// gencore.cuh -- one warp group of Eq. 9, shared by the plain, fused and
// batched kernels.
//
// A warp owns one instance and walks its stream in groups of G = 32*NPT
// numbers; in a group lane j owns the NPT consecutive numbers my0 + 1 ..
// my0 + NPT (my0 = g0 + NPT*j, counted from the start of the run).  Entering
// a group the warp holds M = the message before the group and, per lane,
// sig = the skip just before the lane's first number.  The group:
//   skips     sv_u = sig a^u mod p, u = 1..NPT                      (Eq. 9a)
//   messages  msg_u = M + (skips of lower lanes) + sv_1 + .. + sv_u  (Eq. 6b, 9b)
//             -- the lower-lane sum is an exclusive warp scan mod n
//   encrypt   x_u = msg_u^e mod n by the instance's program          (Eq. 9c)
// and leaves M and sig ready for the next group; R = (x_u+1)/(n+1) (Eq. 9d)
// is formed where it is stored or consumed (real_of).  Numbers past `len` are
// computed but excluded from the sums that carry into later numbers.
//
// The kernels call messages32/64 and encrypt32/64 per group and write the
// state after the run once, after the loop (write_state_after), so that no
// skip or message has to stay in registers through the exponentiation.
#pragma once
#include "arith.cuh"
#include "internal.h"

namespace phprng {

static constexpr unsigned kFullMask = 0xffffffffu;

// One skip step s -> a s mod p (group = false) or one warp group's advance
// s -> a^(32 NPT) s mod p (group = true), as a Montgomery product with the
// constant in Montgomery form.  (A Mersenne fold for p = 2^31 - 1 was measured
// slower on GB300: it trades two multiplier slots for three ALU operations.)
__device__ __forceinline__ uint32_t skip_step(const SkipConst &sk, uint32_t s, bool group)
{
    return group ? mont32c(s, sk.aGM, sk.aGMq, sk.p) : mont32c(s, sk.aM, sk.aMq, sk.p);
}

// The same for a wide skip prime p < 2^63 (Montgomery products mod p, R = 2^64).
__device__ __forceinline__ uint64_t skip_step(const SkipConst64 &sk, uint64_t s, bool group)
{
    return mont64(s, group ? sk.aGM : sk.aM, sk.p, sk.pinv);
}

// s * a^(c Lc) mod p for a plain skip s: the start skip of chunk c of a
// split launch (square-and-multiply on a^Lc in Montgomery form).
__device__ __forceinline__ uint32_t skip_chunk(const SkipConst &sk, const SplitArgs &sp, uint32_t s,
                                               uint32_t c)
{
    uint32_t r = sp.oneM, b = sp.aLcM;
    for (; c; c >>= 1) {
        if (c & 1) r = mont32(r, b, sk.p, sk.pinv);
        b = mont32(b, b, sk.p, sk.pinv);
    }
    return mont32(s, r, sk.p, sk.pinv);
}

// Launch slot w of a split launch: instance slot q = w / K, chunk c = w mod K
// (w < 2^32 whenever K > 1).
__device__ __forceinline__ void split_slot(const SplitArgs &sp, uint64_t w, uint64_t *q, uint32_t *c)
{
    // w / K as the high word of w * ceil(2^64 / K): exact for w < 2^32
    // (the excess w (Kinv - 2^64/K) / 2^64 stays below 2^-32 < 1/K)
    const uint64_t qq = sp.K == 1 ? w : __umul64hi(w, sp.Kinv);
    *q = qq;
    *c = (uint32_t)(w - qq * sp.K);
}

// Start message of chunk c of slot q: the slot's start message plus the skip
// sums of chunks 0 .. c-1, mod n (every lane gets it).
__device__ __forceinline__ uint64_t chunk_message(const SplitArgs &sp, uint64_t q, uint32_t c,
                                                  uint64_t n, int lane)
{
    const uint64_t *h = sp.scratch + q * (sp.K + 1);
    uint64_t S = 0;
    for (uint32_t k = lane; k < c; k += 32) S = addmod64(S, h[2 + k], n);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) S = addmod64(S, __shfl_xor_sync(kFullMask, S, off), n);
    return addmod64(h[0], S, n);
}

// FULL: the whole warp group lies inside the run (no number past len), so
// the per-number bounds checks are left out.
//
// The lane's skip sum and its messages are formed with lazy additions (a
// skip is below p < n): the sum is reduced once before the scan (one
// subtraction when n > 2^31, where every 32-bit value is below 2n), and each
// msg_u is the message mod n up to a multiple of n, a value below 2^32 --
// which the Montgomery products of the encryption accept (their outputs stay
// below 2^32, and the exit product by K < n returns c < n).  M stays reduced.
template <int NPT, bool FULL = false>
__device__ __forceinline__ void messages32(const DevInst &P, const SkipConst &sk, int lane,
                                           uint64_t my0, uint64_t len, uint32_t &M, uint32_t &sig,
                                           uint32_t (&sv)[NPT], uint32_t (&msg)[NPT])
{
    const uint32_t n = (uint32_t)P.n;
    uint32_t S = 0, t = sig;
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        t = skip_step(sk, t, false);                             // Eq. 9a
        sv[u] = t;
        if (FULL || my0 + u < len) S = addmod32_lazy(S, t, n);
    }
    S = (n >> 31) ? (S >= n ? S - n : S) : S % n;
    uint32_t incl = S;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, incl, off);
        if (lane >= off) incl = addmod32(incl, y, n);
    }
    const uint32_t total = __shfl_sync(kFullMask, incl, 31);
    uint32_t mm = addmod32(M, submod32(incl, S, n), n);
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        mm = addmod32_lazy(mm, sv[u], n);                         // Eq. 9b (mod n up to a multiple of n)
        msg[u] = mm;
    }
    M = addmod32(M, total, n);
    sig = skip_step(sk, sig, true);
}

// SK, SW: SkipConst and uint32_t skips (p < 2^32), or SkipConst64 and
// uint64_t skips (a wide skip prime).
template <int NPT, typename SK = SkipConst, typename SW = uint32_t>
__device__ __forceinline__ void messages64(const DevInst &P, const SK &sk, int lane,
                                           uint64_t my0, uint64_t len, uint64_t &M, SW &sig,
                                           SW (&sv)[NPT], uint64_t (&msg)[NPT])
{
    const uint64_t n = P.n;
    uint64_t S = 0;
    SW t = sig;
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        t = skip_step(sk, t, false);
        sv[u] = t;
        if (my0 + u < len) S = addmod64(S, t, n);
    }
    uint64_t incl = S;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(kFullMask, incl, off);
        if (lane >= off) incl = addmod64(incl, y, n);
    }
    const uint64_t total = __shfl_sync(kFullMask, incl, 31);
    uint64_t mm = addmod64(M, incl >= S ? incl - S : incl - S + n, n);
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        mm = addmod64(mm, sv[u], n);
        msg[u] = mm;
    }
    M = addmod64(M, total, n);
    sig = skip_step(sk, sig, true);
}

// Eq. 9c for the lane's NPT messages.  Exponents e = 2^t + 1 (the paper's
// recommended 9 and 17, also 3, 5, 65537) take a straight chain -- t
// squarings and one product with m -- without reading a program; it is the
// chain the host compiles for them, so the exit constant K is the same.
template <int NPT, typename W>
__device__ __forceinline__ void encrypt(const DevInst &P, const ExpProg &pg, const W (&msg)[NPT],
                                        W (&x)[NPT])
{
    const W n = (W)P.n, ninv = (W)P.ninv, K = (W)P.K, Kq = (W)(P.ninv >> 32);
    if (P.fermat) {
        // the first squaring reads the messages directly; the paper's
        // e = 9 and 17 (t = 3, 4) and e = 3, 5 run unrolled chains
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = mont(msg[u], msg[u], n, ninv);
        switch (P.fermat) {
        case 1: break;
        case 2: mont_sqr_vec<NPT>(x, n, ninv); break;
        case 3:
            mont_sqr_vec<NPT>(x, n, ninv);
            mont_sqr_vec<NPT>(x, n, ninv);
            break;
        case 4:
            mont_sqr_vec<NPT>(x, n, ninv);
            mont_sqr_vec<NPT>(x, n, ninv);
            mont_sqr_vec<NPT>(x, n, ninv);
            break;
        default:
            for (uint32_t q = P.fermat; q > 1; --q) mont_sqr_vec<NPT>(x, n, ninv);
            break;
        }
        mont_vec<NPT>(x, msg, n, ninv);
#pragma unroll
        for (int u = 0; u < NPT; ++u) x[u] = mont_exit(x[u], K, Kq, n, ninv);
        return;
    }
    modexp_prog<NPT, W>(x, msg, pg, n, ninv, K, Kq);
}
template <int NPT>
__device__ __forceinline__ void encrypt32(const DevInst &P, const ExpProg &pg, const uint32_t (&msg)[NPT],
                                          uint32_t (&x)[NPT])
{
    encrypt<NPT, uint32_t>(P, pg, msg, x);
}
template <int NPT>
__device__ __forceinline__ void encrypt64(const DevInst &P, const ExpProg &pg, const uint64_t (&msg)[NPT],
                                          uint64_t (&x)[NPT])
{
    encrypt<NPT, uint64_t>(P, pg, msg, x);
}

// The window program of Eq. 9c with its table of odd powers m, m^3, m^5, m^7
// in shared memory instead of registers: per warp 4 entries x NPT values per
// lane, laid out [entry][row][lane] as uint4 rows (four 32-bit or two 64-bit
// values), so that each access of a warp is one conflict-free 512-byte row; a
// lane reads back only its own words, so no synchronisation is needed.  Frees
// 3 NPT values' registers (more resident warps hide the products' latency
// better) for 16-byte loads per window.
template <int NPT, typename W>
__device__ __forceinline__ void put_row(uint4 *__restrict__ tb, int e, int lane, const W (&v)[NPT])
{
    constexpr int Q = NPT * (int)sizeof(W) / 16;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        uint4 w;
        if (sizeof(W) == 4)
            w = make_uint4((uint32_t)v[4 * q], (uint32_t)v[4 * q + 1], (uint32_t)v[4 * q + 2], (uint32_t)v[4 * q + 3]);
        else
            w = make_uint4((uint32_t)v[2 * q], (uint32_t)((uint64_t)v[2 * q] >> 32),
                           (uint32_t)v[2 * q + 1], (uint32_t)((uint64_t)v[2 * q + 1] >> 32));
        tb[(e * Q + q) * 32 + lane] = w;
    }
}

template <int NPT, typename W>
__device__ __forceinline__ void get_row(const uint4 *__restrict__ tb, int e, int lane, W (&v)[NPT])
{
    constexpr int Q = NPT * (int)sizeof(W) / 16;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint4 w = tb[(e * Q + q) * 32 + lane];
        if (sizeof(W) == 4) {
            v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
        } else {
            v[2 * q] = (W)(((uint64_t)w.y << 32) | w.x);
            v[2 * q + 1] = (W)(((uint64_t)w.w << 32) | w.z);
        }
    }
}

template <int NPT, typename W>
__device__ __forceinline__ void modexp_prog_smem(W (&x)[NPT], const W (&m)[NPT], const ExpProg &pg, W n, W ninv,
                                                 W K, W Kq, uint4 *__restrict__ tb, int lane)
{
    static_assert(NPT * sizeof(W) % 16 == 0, "table rows are 16 bytes");
    const int tbl = pg.tbl;
    put_row<NPT, W>(tb, 0, lane, m);
    if (tbl >= 2) {
        W m2[NPT], t[NPT];
#pragma unroll
        for (int u = 0; u < NPT; ++u) m2[u] = mont(m[u], m[u], n, ninv);          // m^2
#pragma unroll
        for (int u = 0; u < NPT; ++u) t[u] = mont(m2[u], m[u], n, ninv);          // m^3
        put_row<NPT, W>(tb, 1, lane, t);
        if (tbl == 4) {
            mont_vec<NPT>(t, m2, n, ninv);                                         // m^5
            put_row<NPT, W>(tb, 2, lane, t);
            mont_vec<NPT>(t, m2, n, ninv);                                         // m^7
            put_row<NPT, W>(tb, 3, lane, t);
        }
    }
    get_row<NPT, W>(tb, pg.ent[0] >> 6, lane, x);
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
        W y[NPT];
        get_row<NPT, W>(tb, b >> 6, lane, y);
        mont_vec<NPT>(x, y, n, ninv);
    }
    for (int sq = pg.tail; sq > 0; --sq) mont_sqr_vec<NPT>(x, n, ninv);
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont_exit(x[u], K, Kq, n, ninv);
}

// Eq. 9c by the exact-search program (ExpProg8), its table of up to
// kProg8MaxTable odd powers in shared memory (tb: kProg8MaxTable * NPT * 4 * 32
// bytes per warp, the same [entry][row][lane] layout as modexp_prog_smem).
template <int NPT>
__device__ __forceinline__ void modexp_prog8_smem(uint32_t (&x)[NPT], const uint32_t (&m)[NPT],
                                                  const ExpProg8 &pg, uint32_t n, uint32_t ninv,
                                                  uint4 *__restrict__ tb, int lane)
{
    const int tbl = pg.tbl;
    put_row<NPT, uint32_t>(tb, 0, lane, m);
    if (tbl >= 2) {
        uint32_t m2[NPT], t[NPT];
#pragma unroll
        for (int u = 0; u < NPT; ++u) m2[u] = mont32(m[u], m[u], n, ninv);          // m^2
#pragma unroll
        for (int u = 0; u < NPT; ++u) t[u] = m[u];
        for (int k = 1; k < tbl; ++k) {                                              // m^(2k+1)
            mont_vec<NPT>(t, m2, n, ninv);
            put_row<NPT, uint32_t>(tb, k, lane, t);
        }
    }
    get_row<NPT, uint32_t>(tb, pg.ent[0] >> 8, lane, x);
    const int nent = pg.nent;
    int bnext = pg.ent[1];
    for (int k = 1; k < nent; ++k) {
        const int b = bnext;
        bnext = pg.ent[k + 1 < 32 ? k + 1 : k];                     // next entry, loaded early
        int sq = b & 0xFF;
        for (; sq >= 2; sq -= 2) {
            mont_sqr_vec<NPT>(x, n, ninv);
            mont_sqr_vec<NPT>(x, n, ninv);
        }
        if (sq) mont_sqr_vec<NPT>(x, n, ninv);
        uint32_t y[NPT];
        get_row<NPT, uint32_t>(tb, (b >> 8) & 7, lane, y);
        mont_vec<NPT>(x, y, n, ninv);
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) x[u] = mont32c(x[u], pg.K, pg.Kq, n);
}

// Eq. 9c for the 32-bit kernels: straight chains for e = 2^t + 1 (no table),
// else the exact-search program with its table at tb (modexp_prog8_smem).
template <int NPT>
__device__ __forceinline__ void encrypt32_p8(const DevInst &P, const ExpProg &pg, const ExpProg8 &pg8,
                                             const uint32_t (&msg)[NPT], uint32_t (&x)[NPT], uint4 *tb, int lane)
{
    if (P.fermat)
        encrypt<NPT, uint32_t>(P, pg, msg, x);
    else
        modexp_prog8_smem<NPT>(x, msg, pg8, (uint32_t)P.n, (uint32_t)P.ninv, tb, lane);
}

// Eq. 9c with the program's table in shared memory (tb: 4 NPT sizeof(W) * 32
// bytes per warp, 16-byte aligned); straight chains need no table.
template <int NPT, typename W>
__device__ __forceinline__ void encrypt_tb(const DevInst &P, const ExpProg &pg, const W (&msg)[NPT], W (&x)[NPT],
                                           uint4 *tb, int lane)
{
    if (P.fermat) {
        encrypt<NPT, W>(P, pg, msg, x);
        return;
    }
    modexp_prog_smem<NPT, W>(x, msg, pg, (W)P.n, (W)P.ninv, (W)P.K, (W)(P.ninv >> 32), tb, lane);
}

template <int NPT>
__device__ __forceinline__ void encrypt32_tb(const DevInst &P, const ExpProg &pg, const uint32_t (&msg)[NPT],
                                             uint32_t (&x)[NPT], uint4 *tb, int lane)
{
    encrypt_tb<NPT, uint32_t>(P, pg, msg, x, tb, lane);
}

// R = (c+1)/(n+1) (Eq. 9d): integer-built and correctly rounded for 32-bit
// n, RN(RN(c+1)/RN(n+1)) by the FP64 unit for 64-bit n.
__device__ __forceinline__ double real_of(const DevInst &P, uint32_t c)
{
    return real32_fast(c, P.yN, P.ybits, P.aux);
}
__device__ __forceinline__ double real_of(const DevInst &P, uint64_t c) { return real64(c, P.n); }

// R of a lane's NPT numbers: every estimate first, without branches (so the
// NPT computations interleave), then, in a lane where some estimate lies in
// the rounding band (one number in about 680), the exact decision for those.
template <int NPT>
__device__ __forceinline__ void reals_of(const DevInst &P, const uint32_t (&x)[NPT], double (&r)[NPT])
{
    uint32_t amb = 0;
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        uint32_t a;
        r[u] = real32_est(x[u], P.yN, P.ybits, P.aux, &a);
        amb |= a << u;
    }
    if (amb) {
#pragma unroll
        for (int u = 0; u < NPT; ++u)
            if ((amb >> u) & 1u) r[u] = real32_exact(x[u], P.yN, P.ybits, P.aux);
    }
}

// Two doubles as one 16-byte store of their four 32-bit words: with R formed
// one number at a time (the LIGHT loop, e = 9: 0.969 -> 0.963 ms) this takes
// one instruction per number fewer than a double2 built from the doubles; the
// pairs formed by reals_of are stored as a double2 (3.812 against 3.805 ms).
__device__ __forceinline__ void store_r2(double *dst, double a, double b)
{
    const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
    *reinterpret_cast<uint4 *>(dst) =
        make_uint4((uint32_t)ba, (uint32_t)(ba >> 32), (uint32_t)bb, (uint32_t)(bb >> 32));
}

// Stores a lane's NPT outputs (16-byte vectors when the whole run of the
// lane is inside `len` and vec_ok says the addresses are aligned).
// RC: numbers whose R are formed together (reals_of; 1: one at a time).
template <int NPT, typename CT, typename XT, bool FULL = false, int RC = 1>
__device__ __forceinline__ void store_group(const DevInst &P, CT *c_dst, double *r_dst,
                                            uint64_t my0, uint64_t len, bool vec_ok,
                                            const XT (&x)[NPT])
{
    const bool full = FULL || my0 + NPT <= len;
    if (c_dst) {
        CT *dst = c_dst + my0;
        if (full && vec_ok && sizeof(CT) == 4 && NPT % 4 == 0) {
#pragma unroll
            for (int u = 0; u < NPT; u += 4)
                *reinterpret_cast<uint4 *>(dst + u) =
                    make_uint4((uint32_t)x[u], (uint32_t)x[u + 1], (uint32_t)x[u + 2], (uint32_t)x[u + 3]);
        } else if (full && vec_ok && sizeof(CT) == 8 && NPT % 2 == 0) {
#pragma unroll
            for (int u = 0; u < NPT; u += 2)
                *reinterpret_cast<ulonglong2 *>(dst + u) = make_ulonglong2(x[u], x[u + 1]);
        } else {
#pragma unroll
            for (int u = 0; u < NPT; ++u)
                if (my0 + u < len) dst[u] = (CT)x[u];
        }
    }
    if (r_dst) {
        double *dst = r_dst + my0;
        if constexpr (sizeof(XT) == 4 && RC > 1 && NPT % RC == 0) {
#pragma unroll
            for (int u0 = 0; u0 < NPT; u0 += RC) {
                XT xc[RC];
                double r[RC];
#pragma unroll
                for (int u = 0; u < RC; ++u) xc[u] = x[u0 + u];
                reals_of<RC>(P, xc, r);
                if (full && vec_ok && RC % 2 == 0) {
#pragma unroll
                    for (int u = 0; u < RC; u += 2)
                        *reinterpret_cast<double2 *>(dst + u0 + u) = make_double2(r[u], r[u + 1]);
                } else {
#pragma unroll
                    for (int u = 0; u < RC; ++u)
                        if (my0 + u0 + u < len) dst[u0 + u] = r[u];
                }
            }
        } else if (full && vec_ok && NPT % 2 == 0) {
#pragma unroll
            for (int u = 0; u < NPT; u += 2) store_r2(dst + u, real_of(P, x[u]), real_of(P, x[u + 1]));
        } else {
#pragma unroll
            for (int u = 0; u < NPT; ++u)
                if (my0 + u < len) dst[u] = real_of(P, x[u]);
        }
    }
}

// The lane that owns number `len` of the run (g0 the group's first index),
// or -1 in the other lanes and groups; u_out = its slot.
template <int NPT>
__device__ __forceinline__ bool owns_last(int lane, uint64_t g0, uint64_t len, int *u_out)
{
    constexpr uint64_t G = 32 * NPT;
    if (g0 + G < len) return false;
    const uint64_t last = len - 1 - g0;
    if ((uint64_t)lane != last / NPT) return false;
    *u_out = (int)(last % NPT);
    return true;
}

// State after the run, before the encryption: message, skip and position.
template <int NPT, typename MT>
__device__ __forceinline__ void write_ms_if_last(DevState st, uint64_t i, int lane, uint64_t g0,
                                                 uint64_t len, uint64_t pos_after,
                                                 const uint32_t (&sv)[NPT], const MT (&msg)[NPT],
                                                 uint64_t n)
{
    int ul;
    if (!owns_last<NPT>(lane, g0, len, &ul)) return;
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        if (u == ul) {
            st.m[i] = (uint64_t)msg[u] % (uint64_t)n;           // 32-bit messages are lazy
            st.s[i] = sv[u];
        }
    }
    st.pos[i] = pos_after;
}

// ... and the last ciphertext, after it.
template <int NPT, typename XT>
__device__ __forceinline__ void write_c_if_last(DevState st, uint64_t i, int lane, uint64_t g0,
                                                uint64_t len, const XT (&x)[NPT])
{
    int ul;
    if (!owns_last<NPT>(lane, g0, len, &ul)) return;
#pragma unroll
    for (int u = 0; u < NPT; ++u)
        if (u == ul) st.c[i] = x[u];
}

// State after a run, written once after the group loop by the lane that owns
// the run's last number: M (the message after the last group, which is the
// last number's message), that number's skip -- sig_group (the lane's skip
// entering the last group, g0) stepped ul+1 times -- and its ciphertext.
template <int NPT, typename XT, typename MT, typename SK = SkipConst, typename SW = uint32_t>
__device__ __forceinline__ void write_state_after(DevState st, const SK &sk, uint64_t i, int lane,
                                                  uint64_t g0, uint64_t len, uint64_t pos_after, MT M,
                                                  SW sig_group, const XT (&x)[NPT])
{
    int ul;
    if (!owns_last<NPT>(lane, g0, len, &ul)) return;
    SW s = sig_group;
    for (int u = 0; u <= ul; ++u) s = skip_step(sk, s, false);
    XT c = x[0];
#pragma unroll
    for (int u = 1; u < NPT; ++u)
        if (u == ul) c = x[u];
    st.m[i] = M;
    st.s[i] = s;
    st.c[i] = c;
    st.pos[i] = pos_after;
}

}  // namespace phprng
