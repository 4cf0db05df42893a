// gen.cu -- generator kernels: Eq. 9 for many independent instances.
//
// One warp owns one instance, so the exponent -- and with it every branch of
// the square-and-multiply program -- is uniform across the warp.  The warp
// walks the instance's stream in groups of 32*NPT numbers (gencore.cuh: skip
// steps, warp scan of the messages, encryption, integer-built R); a group's
// outputs are one contiguous run, so every lane stores 16-byte vectors.  The
// lane that owns the call's last number writes the state back (m, s, c, pos).
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "gencore.cuh"

namespace phprng {

#ifndef PH_MINB32
#define PH_MINB32 3
#endif
#ifndef PH_WPB
#define PH_WPB 8
#endif
static constexpr int kNPT = PH_NPT32;     // numbers per lane per group (32-bit path)
static constexpr int kNPT64 = PH_NPT64;   // numbers per lane per group (64-bit path)
static constexpr int kWarpsPerBlock = PH_WPB;
#ifndef PH_WPB_HEAVY
#define PH_WPB_HEAVY 8
#endif
#ifndef PH_WPB_LIGHT
#define PH_WPB_LIGHT 8
#endif
static constexpr int kWarpsLight = PH_WPB_LIGHT;   // warps per block of the LIGHT instantiation
static constexpr int kWarpsHeavy = PH_WPB_HEAVY;   // warps per block of the plain heavy instantiation (3 blocks of 8 warps per SM, exponent tables in shared memory)
static constexpr unsigned kFull = kFullMask;
// shared memory of one warp's exponent table in the statistics instantiation
// (the standard program: up to 4 odd powers, one 16-byte row per lane and
// NPT/4 numbers each)
static constexpr size_t kTableBytes = 4 * (kNPT / 4) * 32 * sizeof(uint4);
// ... and in the heavy plain instantiation (the exact-search program: up to
// kProg8MaxTable odd powers)
static constexpr size_t kTable8Bytes = kProg8MaxTable * (kNPT / 4) * 32 * sizeof(uint4);
// ... and of a block of the 64-bit launch (kWarpsPerBlock warps, NPT64 values of 8 bytes)
static constexpr size_t kTable64Bytes = (size_t)kWarpsPerBlock * 4 * (kNPT64 / 2) * 32 * sizeof(uint4);

int gen_npt(int wide) { return wide ? kNPT64 : kNPT; }

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 warp_sum_u128(u128 v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const uint64_t lo = __shfl_xor_sync(kFull, (uint64_t)v, off);
        const uint64_t hi = __shfl_xor_sync(kFull, (uint64_t)(v >> 64), off);
        v += ((u128)hi << 64) | lo;
    }
    return v;
}

__device__ __forceinline__ double u128d(u128 v) { return u128_to_double((uint64_t)(v >> 64), (uint64_t)v); }

// STATS = false: the plain generator.  STATS = true: the fused consumer mode
// -- the same numbers, plus per-stream exact sums X = sum(c+1),
// Y = sum(c+1)^2, Z = sum(c+1)(c'+1) with the next instance of the call, and
// a 256-bin histogram of floor(256 R), reduced on chip.  In that mode the
// block's warps walk their groups in lockstep (one block barrier per group):
// each group's ciphertexts go to a double-buffered shared array so a warp can
// pair them with the next warp's; the first and last warp of a block also
// leave their ciphertexts in `edge` so stats_edge_kernel can pair instances
// that straddle two blocks.
#ifndef PH_MINB_STATS
#define PH_MINB_STATS 3
#endif

#ifndef PH_RCHUNK_HEAVY
#define PH_RCHUNK_HEAVY 2
#endif
#ifndef PH_MINB_LIGHT
#define PH_MINB_LIGHT 3
#endif

// LIGHT: the instantiation for launches whose exponent programs are short
// (the paper's small exponents): there the work besides the products (skip
// sums, scan, R, stores) dominates, and three resident blocks per SM with
// the stores of group g placed after group g+1's messages hide it better;
// for long programs two blocks with in-order stores are faster.
template <int NPT, typename CT, bool STATS, bool LIGHT, int WB>
__global__ void __launch_bounds__(WB * 32, STATS ? PH_MINB_STATS : LIGHT ? PH_MINB_LIGHT : PH_MINB32)
gen32_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog,
             const ExpProg8 *__restrict__ prog8, DevState st,
             SkipConst sk, uint64_t first, uint64_t num, uint64_t per_inst,
             CT *__restrict__ c_out, double *__restrict__ r_out, int vec_ok,
             phprng_stats *__restrict__ stats, uint32_t *__restrict__ edge,
             const uint32_t *__restrict__ order, SplitArgs sp)
{
    extern __shared__ __align__(16) uint32_t smem[];   // STATS: cbuf[2][W][32*NPT], hist[W][256], exponent tables; heavy plain: exponent tables
    constexpr int W = WB;
    constexpr uint64_t G = 32 * NPT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // statistics: `order` gives the blocks' launch order (heaviest first); the
    // block keeps its W consecutive instances, which the adjacent-stream
    // products need, and its boundary rows go by its own index lb
    const uint64_t lb = (STATS && order) ? (uint64_t)order[blockIdx.x] : (uint64_t)blockIdx.x;
    const uint64_t w = lb * W + warp;
    // statistics launches are never split (sp.K = 1)
    const bool active = STATS ? w < num : w < num * sp.K;
    if (!STATS && !active) return;
    uint64_t q = w;                                    // instance slot
    uint32_t cidx = 0;                                 // chunk of it
    if (!STATS) split_slot(sp, w, &q, &cidx);
    // the instance this warp runs, relative to `first` (statistics: always w)
    const uint64_t j = !active ? 0 : (!STATS && order) ? order[q] : q;
    const uint64_t i = first + j;
    const DevInst P = inst[i];
    if (!STATS && P.wide) return;
    const ExpProg &pg = prog[i];
    const uint64_t b0 = (uint64_t)cidx * sp.Lc;       // first number of the chunk
    if (!STATS && b0 >= per_inst) return;             // empty trailing chunk
    const uint64_t len = sp.K == 1 ? per_inst : min(sp.Lc, per_inst - b0);
    const bool wb = b0 + len == per_inst;             // the chunk that ends the call

    uint32_t M, sig;
    if (sp.K == 1) {
        M = (uint32_t)st.m[i];
        sig = (uint32_t)st.s[i];
    } else {
        M = (uint32_t)chunk_message(sp, q, cidx, P.n, lane);
        sig = skip_chunk(sk, sp, (uint32_t)sp.scratch[q * (sp.K + 1) + 1], cidx);
    }
    sig = mont32(sig, sk.lane[lane], sk.p, sk.pinv);
    const uint64_t pos_after = wb ? st.pos[i] + per_inst : 0;
    CT *cdst = c_out ? c_out + j * per_inst + b0 : nullptr;
    double *rdst = r_out ? r_out + j * per_inst + b0 : nullptr;

    uint32_t *hist = smem + 2 * W * (32 * NPT) + warp * 256;
    uint64_t X = 0;      // < 2^63: per_inst < 2^31 numbers of at most 2^32 each
    u128 Y = 0, Z = 0;
    const uint32_t binr = (uint32_t)(P.V >> 44);      // floor(2^40 / yN), for the histogram
    const bool has_next = w + 1 < num;
    const bool pair_in_block = has_next && warp + 1 < W;
    if (STATS) {
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
    }

    if constexpr (!STATS) {
        // The plain loop carries nothing but the group step and the stores;
        // the lane that owns the call's last number writes the state after
        // it, once, after the loop.
        uint32_t x[NPT], sig_last = sig;
        uint64_t g_last = 0;
        if (LIGHT) {
            uint32_t xp[NPT];
            uint64_t myp = 0;
            for (uint64_t g0 = 0; g0 < len; g0 += G) {
                uint32_t sv[NPT], msg[NPT];
                const uint64_t my0 = g0 + (uint64_t)NPT * lane;
                sig_last = sig;
                g_last = g0;
                // every group but the last is full: the messages of a full
                // group and the stores of the previous group skip the
                // per-number bounds checks
                if (g0 + G <= len)
                    messages32<NPT, true>(P, sk, lane, my0, len, M, sig, sv, msg);
                else
                    messages32<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
                if (g0) store_group<NPT, CT, uint32_t, true>(P, cdst, rdst, myp, len, vec_ok, xp);
                encrypt32<NPT>(P, pg, msg, x);
#pragma unroll
                for (int u = 0; u < NPT; ++u) xp[u] = x[u];
                myp = my0;
            }
            store_group<NPT, CT, uint32_t>(P, cdst, rdst, myp, len, vec_ok, xp);
        } else {
            // the exponent program's table of up to kProg8MaxTable odd powers
            // lives in shared memory (dynamic, kTable8Bytes per warp)
            uint4 *tb = reinterpret_cast<uint4 *>(smem) + warp * (NPT / 4) * kProg8MaxTable * 32;
            const ExpProg8 &pg8 = prog8[i];
            for (uint64_t g0 = 0; g0 < len; g0 += G) {
                uint32_t sv[NPT], msg[NPT];
                const uint64_t my0 = g0 + (uint64_t)NPT * lane;
                sig_last = sig;
                g_last = g0;
                // full groups skip the per-number bounds checks (fewer
                // instructions and registers)
                const bool full = g0 + G <= len;             // warp-uniform
                if (full)
                    messages32<NPT, true>(P, sk, lane, my0, len, M, sig, sv, msg);
                else
                    messages32<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
                if (P.fermat)
                    encrypt32<NPT>(P, pg, msg, x);
                else
                    modexp_prog8_smem<NPT>(x, msg, pg8, (uint32_t)P.n, (uint32_t)P.ninv, tb, lane);
                // R of two numbers at a time (reals_of)
                if (full)
                    store_group<NPT, CT, uint32_t, true, PH_RCHUNK_HEAVY>(P, cdst, rdst, my0, len, vec_ok, x);
                else
                    store_group<NPT, CT, uint32_t, false, PH_RCHUNK_HEAVY>(P, cdst, rdst, my0, len, vec_ok, x);
            }
        }
        if (wb) write_state_after<NPT, uint32_t, uint32_t>(st, sk, i, lane, g_last, len, pos_after, M,
                                                           sig_last, x);
    } else {
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        uint32_t sv[NPT], msg[NPT], x[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        const bool full = g0 + G <= len;                 // block-uniform (lockstep)
        if (active) {
            if (full)
                messages32<NPT, true>(P, sk, lane, my0, len, M, sig, sv, msg);
            else
                messages32<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
            if (wb) write_ms_if_last<NPT, uint32_t>(st, i, lane, g0, len, pos_after, sv, msg, P.n);
            // the standard program: with the exact-search one (6-entry
            // tables, 80 registers) this loop measured 4.265 against 4.235 ms
            encrypt32_tb<NPT>(P, pg, msg, x,
                              reinterpret_cast<uint4 *>(smem + 2 * W * (32 * NPT) + W * 256) +
                                  warp * (NPT / 4) * 4 * 32,
                              lane);
            store_group<NPT, CT, uint32_t>(P, cdst, rdst, my0, len, vec_ok, x);
            if (wb) write_c_if_last<NPT, uint32_t>(st, i, lane, g0, len, x);
        }
        if (STATS) {
            uint32_t *cb = smem + ((int)((g0 / G) & 1) * W + warp) * (32 * NPT);
            if (active) {
                if (full) {
#pragma unroll
                    for (int u = 0; u < NPT; ++u) {
                        cb[NPT * lane + u] = x[u];
                        const uint64_t v = (uint64_t)x[u] + 1;
                        X += v;
                        Y += (u128)(v * v);
                        atomicAdd(&hist[hist_bin256_int(x[u], P.yN, P.ybits, binr)], 1u);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < NPT; ++u) {
                        cb[NPT * lane + u] = x[u];
                        if (my0 + u < per_inst) {
                            const uint64_t v = (uint64_t)x[u] + 1;
                            X += v;
                            Y += (u128)(v * v);
                            atomicAdd(&hist[hist_bin256_int(x[u], P.yN, P.ybits, binr)], 1u);
                        }
                    }
                }
                if (edge && ((warp == W - 1 && has_next) || (warp == 0 && lb > 0))) {
                    uint32_t *row = edge + (2 * lb + (warp == 0 ? 0 : 1)) * per_inst;
#pragma unroll
                    for (int u = 0; u < NPT; ++u)
                        if (my0 + u < per_inst) row[my0 + u] = x[u];
                }
            }
            // every thread of the block runs the same number of groups, so
            // all of them reach this barrier once per group
            __syncthreads();
            if (active && pair_in_block) {
                const uint32_t *cn = cb + 32 * NPT;              // next warp, same buffer
#pragma unroll
                for (int u = 0; u < NPT; ++u)
                    if (full || my0 + u < per_inst)
                        Z += (u128)(((uint64_t)x[u] + 1) * ((uint64_t)cn[NPT * lane + u] + 1));
            }
        }
    }
    if (STATS && active) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) X += __shfl_xor_sync(kFull, X, off);
        Y = warp_sum_u128(Y);
        Z = warp_sum_u128(Z);
        __syncwarp();
        phprng_stats *o = stats + w;
        for (int b = lane; b < 256; b += 32) o->hist[b] = hist[b];
        if (lane == 0) {
            const u128 N = per_inst, n1 = P.n + 1;
            o->x_lo = X; o->x_hi = 0;
            o->y_lo = (uint64_t)Y; o->y_hi = (uint64_t)(Y >> 64);
            o->z_lo = (uint64_t)Z; o->z_hi = (uint64_t)(Z >> 64);
            o->count = per_inst;
            o->mean = __ddiv_rn(u128d(X), u128d(N * n1));
            o->var = per_inst >= 2 ? __ddiv_rn(u128d(N * Y - (u128)X * X), u128d(N * (N - 1) * n1 * n1))
                                   : 0.0;
            if (pair_in_block) {
                const u128 nn1 = (u128)inst[i + 1].n + 1;
                o->corr = __ddiv_rn(u128d(Z), u128d(N * n1 * nn1));
            } else {
                o->corr = 0.0;                                   // last of the call, or set by the edge kernel
            }
        }
    }
    }   // STATS
}

// Pairs the last instance of block b with the first of block b+1 (one warp
// per pair): Z and corr of that instance from the rows gen32_kernel left in
// `edge`.
__global__ void __launch_bounds__(256)
stats_edge_kernel(const DevInst *__restrict__ inst, const uint32_t *__restrict__ edge,
                  uint64_t first, uint64_t num, uint64_t per_inst, uint64_t nblocks,
                  phprng_stats *__restrict__ stats)
{
    const uint64_t b = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b + 1 >= nblocks) return;
    const uint32_t *L = edge + (2 * b + 1) * per_inst;
    const uint32_t *F = edge + (2 * (b + 1)) * per_inst;
    u128 Z = 0;
    for (uint64_t k = lane; k < per_inst; k += 32)
        Z += (u128)(((uint64_t)L[k] + 1) * ((uint64_t)F[k] + 1));
    Z = warp_sum_u128(Z);
    if (lane == 0) {
        const uint64_t w = b * kWarpsPerBlock + kWarpsPerBlock - 1;     // < num - 1
        phprng_stats *o = stats + w;
        const u128 N = per_inst;
        const u128 n1 = (u128)inst[first + w].n + 1, nn1 = (u128)inst[first + w + 1].n + 1;
        o->z_lo = (uint64_t)Z;
        o->z_hi = (uint64_t)(Z >> 64);
        o->corr = __ddiv_rn(u128d(Z), u128d(N * n1 * nn1));
    }
}

// WSKIP: a wide skip prime (p >= 2^32, SkipConst64 skw, 64-bit skips); such
// launches are never split.
#ifndef PH_MINB64
#define PH_MINB64 3
#endif
template <int NPT, bool WSKIP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, PH_MINB64)
gen64_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog, DevState st,
             SkipConst sk, SkipConst64 skw, uint64_t first, uint64_t num, uint64_t per_inst,
             uint64_t *__restrict__ c_out, double *__restrict__ r_out, int vec_ok,
             const uint32_t *__restrict__ order, SplitArgs sp)
{
    typedef typename std::conditional<WSKIP, uint64_t, uint32_t>::type SW;
    extern __shared__ uint4 tb64[];                   // per warp: the exponent program's odd powers
    constexpr uint64_t G = 32 * NPT;
    const int lane = threadIdx.x & 31;
    const uint64_t w = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= num * sp.K) return;
    uint64_t q;
    uint32_t cidx;
    split_slot(sp, w, &q, &cidx);
    const uint64_t j = order ? order[q] : q;          // instance first + j
    const uint64_t i = first + j;
    const DevInst P = inst[i];
    if (!P.wide) return;
    const ExpProg &pg = prog[i];
    const uint64_t b0 = (uint64_t)cidx * sp.Lc;
    if (b0 >= per_inst) return;
    const uint64_t len = sp.K == 1 ? per_inst : min(sp.Lc, per_inst - b0);
    const bool wb = b0 + len == per_inst;
    uint64_t M;
    SW sig;
    if constexpr (WSKIP) {
        M = st.m[i];
        sig = mont64(st.s[i], skw.lane[lane], skw.p, skw.pinv);
    } else {
        uint32_t s0;
        if (sp.K == 1) {
            M = st.m[i];
            s0 = (uint32_t)st.s[i];
        } else {
            M = chunk_message(sp, q, cidx, P.n, lane);
            s0 = skip_chunk(sk, sp, (uint32_t)sp.scratch[q * (sp.K + 1) + 1], cidx);
        }
        sig = mont32(s0, sk.lane[lane], sk.p, sk.pinv);
    }
    const uint64_t pos_after = wb ? st.pos[i] + per_inst : 0;
    uint64_t *cdst = c_out ? c_out + j * per_inst + b0 : nullptr;
    double *rdst = r_out ? r_out + j * per_inst + b0 : nullptr;
    uint64_t x[NPT];
    SW sig_last = sig;
    uint64_t g_last = 0;
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        SW sv[NPT];
        uint64_t msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        if constexpr (WSKIP)
            messages64<NPT, SkipConst64, uint64_t>(P, skw, lane, my0, len, M, sig, sv, msg);
        else
            messages64<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
        encrypt_tb<NPT, uint64_t>(P, pg, msg, x, tb64 + (threadIdx.x >> 5) * (NPT / 2) * 4 * 32, lane);
        store_group<NPT, uint64_t, uint64_t>(P, cdst, rdst, my0, len, vec_ok, x);
    }
    if (wb) {
        if constexpr (WSKIP)
            write_state_after<NPT, uint64_t, uint64_t, SkipConst64, uint64_t>(st, skw, i, lane, g_last, len,
                                                                              pos_after, M, sig_last, x);
        else
            write_state_after<NPT, uint64_t, uint64_t>(st, sk, i, lane, g_last, len, pos_after, M, sig_last, x);
    }
}

// Pre-pass of a split launch: warp w sums the skips of chunk w % K of slot
// w / K (mod that instance's n; every chunk but the last), and the first warp
// of each slot records the slot's start message and skip (see SplitArgs).
// sk holds the constants of 8 numbers per lane.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
chunk_sums_kernel(const DevInst *__restrict__ inst, DevState st, SkipConst sk, uint64_t first,
                  uint64_t num, uint64_t per_inst, const uint32_t *__restrict__ order, SplitArgs sp,
                  uint64_t *__restrict__ scratch)
{
    constexpr int NPT = 8;
    constexpr uint64_t G = 32 * NPT;
    const int lane = threadIdx.x & 31;
    const uint64_t w = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= num * sp.K) return;
    uint64_t q;
    uint32_t cidx;
    split_slot(sp, w, &q, &cidx);
    const uint64_t i = first + (order ? order[q] : q);
    uint64_t *h = scratch + q * (sp.K + 1);
    const uint32_t s = (uint32_t)st.s[i];
    if (cidx == 0 && lane == 0) {
        h[0] = st.m[i];
        h[1] = s;
    }
    if (cidx + 1 == sp.K) return;                     // no chunk starts after the last
    const uint64_t n = inst[i].n;
    const uint64_t b0 = (uint64_t)cidx * sp.Lc;
    const uint64_t len = b0 >= per_inst ? 0 : min(sp.Lc, per_inst - b0);
    uint32_t sig = mont32(skip_chunk(sk, sp, s, cidx), sk.lane[lane], sk.p, sk.pinv);
    uint64_t S = 0;
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        uint32_t t = sig;
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            t = skip_step(sk, t, false);                  // Eq. 9a
            if (my0 + u < len) S = addmod64(S, t, n);
        }
        sig = skip_step(sk, sig, true);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) S = addmod64(S, __shfl_xor_sync(kFull, S, off), n);
    if (lane == 0) h[2 + cidx] = S;
}

static int check_launch(std::string *err, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string(what) + ": " + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

// Exponent tables above the default 48 KiB of dynamic shared memory need the
// heavy kernel's explicit limit (on the current device), before its launches
// and before the occupancy query that sizes split launches.
static void heavy_smem_limit()
{
    if (kWarpsHeavy * kTable8Bytes <= 48 * 1024) return;
    cudaFuncSetAttribute(gen32_kernel<kNPT, uint32_t, false, false, kWarpsHeavy>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kWarpsHeavy * kTable8Bytes));
    cudaFuncSetAttribute(gen32_kernel<kNPT, uint64_t, false, false, kWarpsHeavy>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kWarpsHeavy * kTable8Bytes));
}

int launch_gen32(const GenArgs &a, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    if (a.stats && a.sp.K != 1) {
        *err = "gen32_kernel: statistics launches are never split";
        return PHPRNG_EINVAL;
    }
    const uint64_t blocks = ((a.num * a.sp.K) + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const uint64_t blocks_heavy = ((a.num * a.sp.K) + kWarpsHeavy - 1) / kWarpsHeavy;
    const uint64_t blocks_light = ((a.num * a.sp.K) + kWarpsLight - 1) / kWarpsLight;
    cudaStream_t s = (cudaStream_t)stream;
    if (a.stats) {
        const size_t smem = (2 * kWarpsPerBlock * 32 * kNPT + kWarpsPerBlock * 256) * sizeof(uint32_t) +
                            kWarpsPerBlock * kTableBytes;
        if (smem > 48 * 1024) {                         // above the default 48 KiB (current device)
            cudaFuncSetAttribute(gen32_kernel<kNPT, uint32_t, true, false, kWarpsPerBlock>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(gen32_kernel<kNPT, uint64_t, true, false, kWarpsPerBlock>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        if (a.c_is_64)
            gen32_kernel<kNPT, uint64_t, true, false, kWarpsPerBlock><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(
                a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, (uint64_t *)a.c_out, a.r_out,
                a.vec_ok, a.stats, a.edge, a.order, a.sp);
        else
            gen32_kernel<kNPT, uint32_t, true, false, kWarpsPerBlock><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(
                a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, (uint32_t *)a.c_out, a.r_out,
                a.vec_ok, a.stats, a.edge, a.order, a.sp);
        int rc = check_launch(err, "gen32_kernel (statistics) launch");
        if (rc != PHPRNG_OK || blocks < 2) return rc;
        stats_edge_kernel<<<(unsigned)((blocks - 1 + 7) / 8), 256, 0, s>>>(
            a.inst, a.edge, a.first, a.num, a.per_inst, blocks, a.stats);
        return check_launch(err, "stats_edge_kernel launch");
    }
#define PH_GEN32_PLAIN(CTY, LT, WB, NB)                                                             \
    gen32_kernel<kNPT, CTY, false, LT, WB><<<(unsigned)(NB), WB * 32, LT ? 0 : WB * kTable8Bytes, s>>>(    \
        a.inst, a.prog, a.prog8, a.st, a.sk, a.first, a.num, a.per_inst, (CTY *)a.c_out, a.r_out, a.vec_ok, \
        nullptr, nullptr, a.order, a.sp)
    if (!a.light) heavy_smem_limit();
    if (a.c_is_64) {
        if (a.light) PH_GEN32_PLAIN(uint64_t, true, kWarpsLight, blocks_light);
        else PH_GEN32_PLAIN(uint64_t, false, kWarpsHeavy, blocks_heavy);
    } else {
        if (a.light) PH_GEN32_PLAIN(uint32_t, true, kWarpsLight, blocks_light);
        else PH_GEN32_PLAIN(uint32_t, false, kWarpsHeavy, blocks_heavy);
    }
#undef PH_GEN32_PLAIN
    return check_launch(err, "gen32_kernel launch");
}

uint32_t gen32_stats_block_warps() { return kWarpsPerBlock; }

uint64_t gen32_edge_words(uint64_t num, uint64_t per_inst)
{
    const uint64_t blocks = (num + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return blocks < 2 ? 0 : 2 * blocks * per_inst;
}

int launch_gen64(const GenArgs &a, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    const uint64_t blocks = ((a.num * a.sp.K) + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (a.wide_skip) {
        if (a.sp.K != 1) {
            *err = "gen64_kernel: launches with a wide skip prime are never split";
            return PHPRNG_EINVAL;
        }
        gen64_kernel<kNPT64, true><<<(unsigned)blocks, kWarpsPerBlock * 32, kTable64Bytes, (cudaStream_t)stream>>>(
            a.inst, a.prog, a.st, a.sk, a.skw, a.first, a.num, a.per_inst, (uint64_t *)a.c_out, a.r_out,
            a.vec_ok, a.order, a.sp);
    } else {
        gen64_kernel<kNPT64, false><<<(unsigned)blocks, kWarpsPerBlock * 32, kTable64Bytes, (cudaStream_t)stream>>>(
            a.inst, a.prog, a.st, a.sk, a.skw, a.first, a.num, a.per_inst, (uint64_t *)a.c_out, a.r_out,
            a.vec_ok, a.order, a.sp);
    }
    return check_launch(err, "gen64_kernel launch");
}

int launch_chunk_sums(const GenArgs &a, const SkipConst &sk8, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0 || a.sp.K < 2) return PHPRNG_OK;
    const uint64_t blocks = ((a.num * a.sp.K) + kWarpsPerBlock - 1) / kWarpsPerBlock;
    chunk_sums_kernel<<<(unsigned)blocks, kWarpsPerBlock * 32, 0, (cudaStream_t)stream>>>(
        a.inst, a.st, sk8, a.first, a.num, a.per_inst, a.order, a.sp, (uint64_t *)a.sp.scratch);
    return check_launch(err, "chunk_sums_kernel launch");
}

uint64_t gen_resident_warps()
{
    static std::mutex mu;
    static uint64_t cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!cached[dev]) {
        int sms = 0, b = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        heavy_smem_limit();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gen32_kernel<kNPT, uint32_t, false, false, kWarpsHeavy>,
                                                      kWarpsHeavy * 32, kWarpsHeavy * kTable8Bytes);
        cached[dev] = (uint64_t)(sms > 0 ? sms : 1) * (b > 0 ? b : 1) * kWarpsHeavy;
    }
    return cached[dev];
}

// ---- fused statistics with fixed scratch ------------------------------------
// Some callers cannot allocate GPU memory at the point where they want the
// statistics: a caching allocator may already own all device memory, the call
// may sit on a latency-critical path where an allocation would synchronise the
// device, or the code may run where allocation is forbidden after start-up.
// For them the statistics call can use this fixed array for its only scratch
// (the ciphertext rows that pair instances across thread blocks) instead of a
// stream-ordered allocation.  The array lives for as long as the library is
// loaded, on every device that loads it.  Every call shares it and leaves its
// rows behind; each row is written in full before it is read, so nothing needs
// clearing, but two such calls that overlap on the GPU (different streams,
// not ordered) race on it.
static constexpr uint64_t kFixedEdgeWords = 1ull << 20;      // 4 MiB of uint32
static __device__ __align__(256) uint32_t g_fixed_edge[kFixedEdgeWords];

static uint32_t *g_fixed_edge_addr[64];                     // device address, per device
static std::mutex g_fixed_edge_mu;

uint64_t gen32_fixed_edge_words() { return kFixedEdgeWords; }

// The host name g_fixed_edge is only a stand-in for the device array: its
// device address is looked up once per device, with that device current, and
// kept for the process (it is the primary context's; a cudaDeviceReset of the
// device would leave it stale, so the library is not used past one).
static int fixed_edge_address(int dev, uint32_t **out, std::string *err)
{
    if (dev < 0 || dev >= 64) {
        *err = "device index above 63";
        return PHPRNG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_fixed_edge_mu);
    if (!g_fixed_edge_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_edge);
        if (e != cudaSuccess) {
            *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return PHPRNG_ECUDA;
        }
        g_fixed_edge_addr[dev] = (uint32_t *)p;
    }
    *out = g_fixed_edge_addr[dev];
    return PHPRNG_OK;
}

int launch_gen32_stats_fixed(const GenArgs &a, int dev, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    if (gen32_edge_words(a.num, a.per_inst) > kFixedEdgeWords) {
        *err = "statistics scratch of " + std::to_string(gen32_edge_words(a.num, a.per_inst)) +
               " words exceeds the fixed 1,048,576 words (2 x ceil(num_inst/8) x per_inst must "
               "not exceed 2^20)";
        return PHPRNG_EINVAL;
    }
    uint32_t *edge = nullptr;
    int rc = fixed_edge_address(dev, &edge, err);
    if (rc != PHPRNG_OK) return rc;
    GenArgs b = a;
    b.edge = edge;
    return launch_gen32(b, stream, err);
}

}  // namespace phprng
