// skip.cu -- the prefix table of the skip cycle and the skip-ahead kernel.
//
// Table build (once per context, on the device):
//   segments: thread j sums the B consecutive terms a^(jB+1) .. a^((j+1)B)
//             (Eq. 6b with s0 = 1) and records P[j] = a^(jB) mod p;
//   scan:     one block turns the segment sums into T[j] = Pref(jB), exact
//             64-bit prefix sums (every T[j] <= p(p-1)/2 < 2^63).
// Skip kernel: one warp per (instance, k) request evaluates Eq. 7 from the
// instance's current state; the cycle position of its skip is
// L = (L0 + pos) mod (p-1), L0 the discrete log of s0 found on the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "skipdev.cuh"

namespace phprng {

// a^k mod p (plain) by square-and-multiply on Montgomery products.
__device__ __forceinline__ uint32_t pow_a(const SkipTable &tb, uint64_t k)
{
    uint32_t x = tb.oneM;
    for (int b = 63 - __clzll((long long)(k | 1)); b >= 0; --b) {
        x = mont32(x, x, tb.p, tb.pinv);
        if ((k >> b) & 1ull) x = mont32(x, tb.aM, tb.p, tb.pinv);
    }
    return mont32(x, 1u, tb.p, tb.pinv);
}

__global__ void __launch_bounds__(256)
skip_table_segments(SkipTable tb, uint64_t nseg, uint64_t *seg, uint32_t *P)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > nseg) return;
    uint32_t x = pow_a(tb, j << kSkipLog2B);
    P[j] = x;
    if (j == nseg) return;                     // last checkpoint: power only
    uint64_t sum = 0;
#pragma unroll 8
    for (uint32_t u = 0; u < kSkipB; ++u) {
        x = mont32(x, tb.aM, tb.p, tb.pinv);
        sum += x;
    }
    seg[j] = sum;
}

// T[0] = 0, T[j+1] = T[j] + seg[j]; one block of 1024 threads, each owning a
// contiguous run of segments.
__global__ void __launch_bounds__(1024)
skip_table_scan(const uint64_t *seg, uint64_t nseg, uint64_t *T)
{
    __shared__ uint64_t part[1024];
    const uint64_t per = (nseg + 1023) / 1024;
    const uint64_t lo = threadIdx.x * per, hi = min(nseg, lo + per);
    uint64_t s = 0;
    for (uint64_t j = lo; j < hi; ++j) s += seg[j];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    if (threadIdx.x == 0) T[0] = 0;
    for (uint64_t j = lo; j < hi; ++j) {
        run += seg[j];
        T[j + 1] = run;
    }
}

__global__ void __launch_bounds__(256)
skip_kernel(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog, DevState st,
            const uint64_t *__restrict__ L0,
            SkipTable tb, const SkipReq *__restrict__ reqs, uint64_t cnt)
{
    const uint64_t w = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w >= cnt) return;
    const SkipReq q = reqs[w];
    if (q.k == 0) return;
    const uint64_t i = q.inst;
    const DevInst P = inst[i];
    const uint64_t pm1 = tb.p - 1;
    const uint64_t pos = st.pos[i];
    // kind 0: the cycle position of the current skip; kind 1: the constant b
    const uint64_t L = tb.kind == 1 ? L0[i] : (L0[i] + pos % pm1) % pm1;
    uint64_t m;
    uint32_t s;
    uint64_t Lnew;
    if (!q.back) {
        skip_state_warp(tb, P, st.m[i], L, q.k, &m, &s, &Lnew);
    } else if (tb.kind == 1) {
        // backward by k over a constant skip: m' = m - k b mod n, s' = b
        uint64_t F, Lf;
        skip_state_warp(tb, P, 0, L, q.k, &F, &s, &Lf);
        const uint64_t mc = st.m[i];
        m = mc >= F ? mc - F : mc + (P.n - F);
    } else {
        // Backward by k: the state k steps earlier sits at cycle position
        // L' = L - k mod (p-1), and going forward k steps from it adds F =
        // q p(p-1)/2 + (window sum from L') (Eq. 7), so m' = m - F mod n and
        // s' = a^L'.
        Lnew = (L + pm1 - q.k % pm1) % pm1;
        uint64_t F, Lf, sumL;
        uint32_t sf;
        skip_state_warp(tb, P, 0, Lnew, q.k, &F, &sf, &Lf);
        pref_warp(tb, Lnew, &sumL, &s);
        const uint64_t mc = st.m[i];
        m = mc >= F ? mc - F : mc + (P.n - F);
    }
    const uint64_t pos_new = q.back ? pos - q.k : pos + q.k;
    if ((threadIdx.x & 31) == 0) {
        uint64_t c;
        if (!P.wide) {
            uint32_t msg[1] = {(uint32_t)m}, x[1];
            modexp_prog<1, uint32_t>(x, msg, prog[i], (uint32_t)P.n, (uint32_t)P.ninv,
                                     (uint32_t)P.K, (uint32_t)(P.ninv >> 32));
            c = x[0];
        } else {
            uint64_t msg[1] = {m}, x[1];
            modexp_prog<1, uint64_t>(x, msg, prog[i], P.n, P.ninv, P.K, 0);
            c = x[0];
        }
        st.m[i] = m;
        st.s[i] = s;
        st.c[i] = pos_new ? c : 0;                     // Eq. 7c at the new position (0 before
        st.pos[i] = pos_new;                           // the first number)
    }
}

// ---- wide skip primes (p >= 2^32): window sums by parallel stepping ----------

// base^k in Montgomery form from baseM = base 2^64 mod p (square-and-multiply).
__device__ __forceinline__ uint64_t pow64M(const SkipConst64 &sk, uint64_t baseM, uint64_t k)
{
    uint64_t x = sk.oneM;
    for (int b = 63 - __clzll((long long)(k | 1)); b >= 0; --b) {
        x = mont64(x, x, sk.p, sk.pinv);
        if ((k >> b) & 1ull) x = mont64(x, baseM, sk.p, sk.pinv);
    }
    return x;
}

// scratch[0] = the skip the window starts from: s, or s a^-r going back r.
__global__ void wide_skip_prep(DevState st, SkipConst64 sk, uint64_t ainvM, uint64_t inst, uint64_t r,
                               uint64_t back, uint64_t *scratch)
{
    if (threadIdx.x != 0) return;
    const uint64_t s = st.s[inst];
    scratch[0] = back ? mont64(s, pow64M(sk, ainvM, r), sk.p, sk.pinv) : s;
}

// sum_{j=1..r} (sb a^j mod p) mod n, cut into one contiguous run of terms per
// thread (each starts at sb a^(j0+1) by square-and-multiply), reduced per
// block into scratch[1 + block].
__global__ void __launch_bounds__(256)
wide_skip_sum(const DevInst *__restrict__ inst, SkipConst64 sk, uint64_t i, uint64_t r, uint64_t *scratch)
{
    __shared__ uint64_t part[8];
    const uint64_t n = inst[i].n;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t per = (r + T - 1) / T;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t j0 = t * per;
    uint64_t sum = 0;
    if (j0 < r) {
        const uint64_t sb = scratch[0];
        uint64_t v = mont64(sb, pow64M(sk, sk.aM, j0 + 1), sk.p, sk.pinv);   // sb a^(j0+1)
        const uint64_t cnt = min(per, r - j0);
        for (uint64_t u = 0; u < cnt; ++u) {
            sum = addmod64(sum, v, n);                                     // v < p < n
            v = mont64(v, sk.aM, sk.p, sk.pinv);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum = addmod64(sum, __shfl_xor_sync(0xffffffffu, sum, off), n);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = addmod64(b, part[w], n);
        scratch[1 + blockIdx.x] = b;
    }
}

// The state after the piece: F = q p(p-1)/2 + window sum (mod n), m' = m + F
// or m - F, s' = sb a^r or sb, c' = m'^e (0 at position 0), pos' = pos +- k.
__global__ void wide_skip_final(const DevInst *__restrict__ inst, const ExpProg *__restrict__ prog, DevState st,
                                SkipConst64 sk, uint64_t i, uint64_t q, uint64_t r, uint64_t k, uint64_t back,
                                uint64_t nblocks, const uint64_t *scratch)
{
    const int lane = threadIdx.x & 31;
    const DevInst P = inst[i];
    const uint64_t n = P.n;
    uint64_t F = 0;
    for (uint64_t b = lane; b < nblocks; b += 32) F = addmod64(F, scratch[1 + b], n);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) F = addmod64(F, __shfl_xor_sync(0xffffffffu, F, off), n);
    if (lane != 0) return;
    if (q) {
        typedef unsigned __int128 u128;
        const uint64_t half = (uint64_t)((((u128)sk.p * (sk.p - 1)) >> 1) % n);
        F = addmod64(F, (uint64_t)(((u128)(q % n) * half) % n), n);
    }
    const uint64_t sb = scratch[0], m = st.m[i];
    const uint64_t m2 = back ? (m >= F ? m - F : m + (n - F)) : addmod64(m, F, n);
    const uint64_t s2 = back ? sb : mont64(sb, pow64M(sk, sk.aM, r), sk.p, sk.pinv);
    const uint64_t pos2 = back ? st.pos[i] - k : st.pos[i] + k;
    uint64_t msg[1] = {m2}, x[1];
    modexp_prog<1, uint64_t>(x, msg, prog[i], n, P.ninv, P.K, 0);
    st.m[i] = m2;
    st.s[i] = s2;
    st.c[i] = pos2 ? x[0] : 0;
    st.pos[i] = pos2;
}

static int check(std::string *err, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string(what) + ": " + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_build_skip_table(uint64_t p, uint64_t a, uint64_t *T, uint32_t *P, uint64_t *seg,
                            void *stream, std::string *err)
{
    SkipTable tb = derive_skip_table(p, a);
    const uint64_t nseg = tb.nT - 1;
    cudaStream_t s = (cudaStream_t)stream;
    skip_table_segments<<<(unsigned)((nseg + 1 + 255) / 256), 256, 0, s>>>(tb, nseg, seg, P);
    int rc = check(err, "skip_table_segments launch");
    if (rc != PHPRNG_OK) return rc;
    skip_table_scan<<<1, 1024, 0, s>>>(seg, nseg, T);
    return check(err, "skip_table_scan launch");
}

int launch_skip(const DevInst *inst, const ExpProg *prog, DevState st, const uint64_t *L0,
                SkipTable tbl, const SkipReq *reqs, uint64_t cnt, void *stream, std::string *err)
{
    if (cnt == 0) return PHPRNG_OK;
    skip_kernel<<<(unsigned)((cnt + 7) / 8), 256, 0, (cudaStream_t)stream>>>(inst, prog, st, L0,
                                                                               tbl, reqs, cnt);
    return check(err, "skip_kernel launch");
}

}  // namespace phprng

namespace phprng {

// One wide-skip request: r = k mod (p-1) steps in pieces of at most
// kWideSkipPiece, the q full cycles added with the first piece.
int launch_skip_wide(const DevInst *inst, const ExpProg *prog, DevState st, const SkipConst64 &skw,
                     uint64_t ainvM, const SkipReq &req, uint64_t *scratch, void *stream, std::string *err)
{
    if (req.k == 0) return PHPRNG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t pm1 = skw.p - 1;
    const uint64_t q = req.k / pm1, r = req.k % pm1;
    uint64_t done = 0;
    bool first = true;
    do {
        const uint64_t piece = std::min<uint64_t>(r - done, kWideSkipPiece);
        const uint64_t k_piece = first ? q * pm1 + piece : piece;   // positions this piece moves
        const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>(kWideSkipBlocks, (piece + 255) / 256));
        wide_skip_prep<<<1, 32, 0, s>>>(st, skw, ainvM, req.inst, piece, req.back, scratch);
        int rc = check(err, "wide_skip_prep launch");
        if (rc != PHPRNG_OK) return rc;
        wide_skip_sum<<<(unsigned)blocks, 256, 0, s>>>(inst, skw, req.inst, piece, scratch);
        rc = check(err, "wide_skip_sum launch");
        if (rc != PHPRNG_OK) return rc;
        wide_skip_final<<<1, 32, 0, s>>>(inst, prog, st, skw, req.inst, first ? q : 0, piece, k_piece,
                                         req.back, blocks, scratch);
        rc = check(err, "wide_skip_final launch");
        if (rc != PHPRNG_OK) return rc;
        done += piece;
        first = false;
    } while (done < r);
    return PHPRNG_OK;
}

}  // namespace phprng
