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
    const uint64_t L = (L0[i] + pos % pm1) % pm1;
    uint64_t m;
    uint32_t s;
    uint64_t Lnew;
    if (!q.back) {
        skip_state_warp(tb, P, st.m[i], L, q.k, &m, &s, &Lnew);
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
