// gen.cu -- generator kernels: Eq. 9 for many independent instances.
//
// Work split.  One warp owns one instance (its exponent e is then uniform
// across the warp, so the square-and-multiply loop has no divergence).  The
// warp walks the instance's stream in groups of G = 32*NPT numbers; in a
// group lane j owns the NPT consecutive numbers G*g + NPT*j + 1 .. + NPT,
// which makes a lane's outputs contiguous and a group's outputs one
// contiguous run of G values.
//
// Per group (position t before the group, state m_t, s_t):
//   skips   lane j keeps sigma_j = s at the position just before its run and
//           steps it NPT times with Eq. 9a (Montgomery product mod p);
//           sigma_j advances by a^G per group (Eq. 6a: s_k = s_0 a^k mod p);
//   messages  m at lane j's u-th number = m_t + (sum of the skips before it),
//           Eq. 6b, formed as an exclusive warp scan mod n of the lanes'
//           skip sums plus the lane's own running sum (Eq. 9b);
//   encrypt c = m^e mod n (Eq. 9c) by left-to-right square-and-multiply on
//           Montgomery products started from the plain message, closed by
//           one product with the per-instance constant K;
//   float   R = (c+1)/(n+1) (Eq. 9d): integer-built correctly rounded double
//           for n < 2^32, hardware FP64 division of the rounded operands for
//           64-bit n;
//   store   c and/or R; 16-byte vector stores when aligned.
// The lane that owns the last number writes the state back (m, s, c, pos).
#include <cuda_runtime.h>

#include "arith.cuh"
#include "internal.h"

namespace phprng {

static constexpr int kNPT = 4;          // numbers per lane per group (32-bit path)
static constexpr int kNPT64 = 2;        // numbers per lane per group (64-bit path)
static constexpr int kWarpsPerBlock = 8;
static constexpr unsigned kFull = 0xffffffffu;

int gen_npt(int wide) { return wide ? kNPT64 : kNPT; }

template <int NPT, typename CT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
gen32_kernel(const DevInst *__restrict__ inst, DevState st, SkipConst sk, uint64_t first,
             uint64_t num, uint64_t per_inst, CT *__restrict__ c_out,
             double *__restrict__ r_out, int vec_ok)
{
    const int lane = threadIdx.x & 31;
    const uint64_t w = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= num) return;
    const uint64_t i = first + w;
    const DevInst P = inst[i];
    if (P.wide) return;
    const uint32_t n = (uint32_t)P.n, ninv = (uint32_t)P.ninv, K = (uint32_t)P.K;
    const uint32_t e = (uint32_t)P.e;
    const int ebits = (int)P.ebits;
    const uint32_t p = sk.p, pinv = sk.pinv, aM = sk.aM;

    uint32_t M = (uint32_t)st.m[i];
    uint32_t sig = mont32((uint32_t)st.s[i], sk.lane[lane], p, pinv);
    const uint64_t base = w * per_inst;
    constexpr uint64_t G = 32 * NPT;

    for (uint64_t g0 = 0; g0 < per_inst; g0 += G) {
        uint32_t sv[NPT], msg[NPT], x[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        uint32_t S = 0, t = sig;
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            t = mont32(t, aM, p, pinv);                          // Eq. 9a
            sv[u] = t;
            if (my0 + u < per_inst) S = addmod32(S, t, n);
        }
        uint32_t incl = S;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl = addmod32(incl, y, n);
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        uint32_t mm = addmod32(M, submod32(incl, S, n), n);
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            mm = addmod32(mm, sv[u], n);                          // Eq. 9b
            msg[u] = mm;
        }
        modexp32<NPT>(x, msg, e, ebits, n, ninv, K);             // Eq. 9c

        const bool full = my0 + NPT <= per_inst;
        if (c_out) {
            CT *dst = c_out + base + my0;
            if (full && vec_ok && sizeof(CT) == 4 && NPT % 4 == 0) {
#pragma unroll
                for (int u = 0; u < NPT; u += 4)
                    *reinterpret_cast<uint4 *>(dst + u) = make_uint4(x[u], x[u + 1], x[u + 2], x[u + 3]);
            } else if (full && vec_ok && sizeof(CT) == 8 && NPT % 2 == 0) {
#pragma unroll
                for (int u = 0; u < NPT; u += 2)
                    *reinterpret_cast<ulonglong2 *>(dst + u) = make_ulonglong2(x[u], x[u + 1]);
            } else {
#pragma unroll
                for (int u = 0; u < NPT; ++u)
                    if (my0 + u < per_inst) dst[u] = (CT)x[u];
            }
        }
        if (r_out) {
            double *dst = r_out + base + my0;
            double rv[NPT];
#pragma unroll
            for (int u = 0; u < NPT; ++u) rv[u] = real32(x[u], P.yN, P.ybits, P.V);   // Eq. 9d
            if (full && vec_ok && NPT % 2 == 0) {
#pragma unroll
                for (int u = 0; u < NPT; u += 2)
                    *reinterpret_cast<double2 *>(dst + u) = make_double2(rv[u], rv[u + 1]);
            } else {
#pragma unroll
                for (int u = 0; u < NPT; ++u)
                    if (my0 + u < per_inst) dst[u] = rv[u];
            }
        }
        if (g0 + G >= per_inst) {                                // state write-back
            const uint64_t last = per_inst - 1 - g0;
            if ((uint64_t)lane == last / NPT) {
                const int ul = (int)(last % NPT);
#pragma unroll
                for (int u = 0; u < NPT; ++u) {
                    if (u == ul) {
                        st.m[i] = msg[u];
                        st.s[i] = sv[u];
                        st.c[i] = x[u];
                    }
                }
                st.pos[i] += per_inst;
            }
        }
        M = addmod32(M, total, n);
        sig = mont32(sig, sk.aGM, p, pinv);
    }
}

template <int NPT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
gen64_kernel(const DevInst *__restrict__ inst, DevState st, SkipConst sk, uint64_t first,
             uint64_t num, uint64_t per_inst, uint64_t *__restrict__ c_out,
             double *__restrict__ r_out, int vec_ok)
{
    const int lane = threadIdx.x & 31;
    const uint64_t w = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (w >= num) return;
    const uint64_t i = first + w;
    const DevInst P = inst[i];
    if (!P.wide) return;
    const uint64_t n = P.n, ninv = P.ninv, K = P.K, e = P.e;
    const int ebits = (int)P.ebits;
    const uint32_t p = sk.p, pinv = sk.pinv, aM = sk.aM;

    uint64_t M = st.m[i];
    uint32_t sig = mont32((uint32_t)st.s[i], sk.lane[lane], p, pinv);
    const uint64_t base = w * per_inst;
    constexpr uint64_t G = 32 * NPT;

    for (uint64_t g0 = 0; g0 < per_inst; g0 += G) {
        uint32_t sv[NPT];
        uint64_t msg[NPT], x[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        uint64_t S = 0;
        uint32_t t = sig;
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            t = mont32(t, aM, p, pinv);
            sv[u] = t;
            if (my0 + u < per_inst) S = addmod64(S, t, n);
        }
        uint64_t incl = S;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint64_t y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl = addmod64(incl, y, n);
        }
        const uint64_t total = __shfl_sync(kFull, incl, 31);
        uint64_t mm = addmod64(M, incl >= S ? incl - S : incl - S + n, n);
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            mm = addmod64(mm, sv[u], n);                          // Eq. 9b
            msg[u] = mm;
        }
        modexp64<NPT>(x, msg, e, ebits, n, ninv, K);             // Eq. 9c

        const bool full = my0 + NPT <= per_inst;
        if (c_out) {
            uint64_t *dst = c_out + base + my0;
            if (full && vec_ok && NPT % 2 == 0) {
#pragma unroll
                for (int u = 0; u < NPT; u += 2)
                    *reinterpret_cast<ulonglong2 *>(dst + u) = make_ulonglong2(x[u], x[u + 1]);
            } else {
#pragma unroll
                for (int u = 0; u < NPT; ++u)
                    if (my0 + u < per_inst) dst[u] = x[u];
            }
        }
        if (r_out) {
            double *dst = r_out + base + my0;
            double rv[NPT];
#pragma unroll
            for (int u = 0; u < NPT; ++u) rv[u] = real64(x[u], n);
            if (full && vec_ok && NPT % 2 == 0) {
#pragma unroll
                for (int u = 0; u < NPT; u += 2)
                    *reinterpret_cast<double2 *>(dst + u) = make_double2(rv[u], rv[u + 1]);
            } else {
#pragma unroll
                for (int u = 0; u < NPT; ++u)
                    if (my0 + u < per_inst) dst[u] = rv[u];
            }
        }
        if (g0 + G >= per_inst) {
            const uint64_t last = per_inst - 1 - g0;
            if ((uint64_t)lane == last / NPT) {
                const int ul = (int)(last % NPT);
#pragma unroll
                for (int u = 0; u < NPT; ++u) {
                    if (u == ul) {
                        st.m[i] = msg[u];
                        st.s[i] = sv[u];
                        st.c[i] = x[u];
                    }
                }
                st.pos[i] += per_inst;
            }
        }
        M = addmod64(M, total, n);
        sig = mont32(sig, sk.aGM, p, pinv);
    }
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

int launch_gen32(const GenArgs &a, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    const uint64_t blocks = (a.num + kWarpsPerBlock - 1) / kWarpsPerBlock;
    cudaStream_t s = (cudaStream_t)stream;
    if (a.c_is_64)
        gen32_kernel<kNPT, uint64_t><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(
            a.inst, a.st, a.sk, a.first, a.num, a.per_inst, (uint64_t *)a.c_out, a.r_out, a.vec_ok);
    else
        gen32_kernel<kNPT, uint32_t><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(
            a.inst, a.st, a.sk, a.first, a.num, a.per_inst, (uint32_t *)a.c_out, a.r_out, a.vec_ok);
    return check_launch(err, "gen32_kernel launch");
}

int launch_gen64(const GenArgs &a, void *stream, std::string *err)
{
    if (a.num == 0 || a.per_inst == 0) return PHPRNG_OK;
    const uint64_t blocks = (a.num + kWarpsPerBlock - 1) / kWarpsPerBlock;
    gen64_kernel<kNPT64><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, (cudaStream_t)stream>>>(
        a.inst, a.st, a.sk, a.first, a.num, a.per_inst, (uint64_t *)a.c_out, a.r_out, a.vec_ok);
    return check_launch(err, "gen64_kernel launch");
}

}  // namespace phprng
