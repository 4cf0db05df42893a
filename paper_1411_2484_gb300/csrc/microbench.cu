// microbench.cu -- throughput of the units the generator is bound by.
//
// Each kernel runs eight independent dependency chains per thread of one
// instruction form, written in inline PTX so the compiler keeps every
// operation, over a grid that fills every SM at full occupancy; the rate is
// (threads x chains x operations) / elapsed time (CUDA events).
//   0  mul.lo.u32              one 32-bit product half per operation
//   1  mad.hi.u32              one half per operation
//   2  mad.wide.u32            two halves per operation
//   3  Montgomery product mod a 32-bit prime (the generator's mulmod)
//   4  fma.rn.f64              FP64 fused multiply-add
//   5  the generator's window exponent programs alone (Eq. 9c without the
//      skips, scan, R and stores): 65,536 seeded 32-bit instances (safe
//      primes, random exponents), one warp per instance, 8 messages per
//      lane, 16 exponentiations back to back; the rate counts Montgomery
//      products (table, windows, squarings and the exit product).
//   6  div.rn.f64              FP64 division, IEEE round to nearest (what
//                              R = (c+1)/(n+1) costs as a floating division)
//   7  the generator's R built from integers (Eq. 9d, correctly rounded),
//      for n = 2^32 - 5: the replacement of form 6
//   8  mul.wide.u32               both halves of a 32x32 product
//   9  Montgomery product with the low and high halves of a b taken by
//      mul.lo and mul.hi instead of one mul.wide
//  10  Montgomery product by a constant (three multiplies, the constant's
//      q factor precomputed: the generator's exit and skip products)
//  11  product by a constant mod p < 2^31 with a precomputed quotient factor
//      (Shoup): q = hi(x w), x b - q p, one conditional subtraction
#include <cuda_runtime.h>

#include <vector>

#include "arith.cuh"
#include "internal.h"

namespace phprng {

static constexpr int kChains = 8, kUnroll = 16;

template <int FORM>
__global__ void __launch_bounds__(256) microbench_kernel(uint32_t *sink, int iters, uint32_t c,
                                                         uint32_t n, uint32_t ninv, uint32_t yN,
                                                         uint32_t ybits, uint64_t W)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[kChains];
    uint64_t acc[kChains];
    double d[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        x[k] = tid * 2654435761u + k * 40503u + 1u;
        acc[k] = x[k];
        d[k] = 1.0 + 1e-9 * (double)(x[k] & 1023u);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (FORM == 0) {
                    asm volatile("mul.lo.u32 %0, %0, %1;" : "+r"(x[k]) : "r"(c));
                } else if (FORM == 1) {
                    asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(c), "r"(n));
                } else if (FORM == 2) {
                    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[k]) : "r"(x[k]), "r"(c));
                    x[k] = (uint32_t)acc[k];
                } else if (FORM == 3) {
                    x[k] = mont32(x[k], x[k], n, ninv);   // exact for any inputs < 2^32 here
                } else if (FORM == 6) {
                    asm volatile("div.rn.f64 %0, %1, %0;" : "+d"(d[k]) : "d"(1.0000001));
                } else if (FORM == 8) {
                    uint64_t t;
                    asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(t) : "r"(x[k]), "r"(c));
                    x[k] = (uint32_t)t ^ (uint32_t)(t >> 32);
                } else if (FORM == 9) {
                    uint32_t lo, hi, q, u;
                    asm volatile("mul.lo.u32 %0, %1, %1;" : "=r"(lo) : "r"(x[k]));
                    asm volatile("mul.hi.u32 %0, %1, %1;" : "=r"(hi) : "r"(x[k]));
                    asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(q) : "r"(lo), "r"(ninv));
                    asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(u) : "r"(q), "r"(n));
                    const uint32_t t = hi - u;
                    x[k] = hi < u ? t + n : t;
                } else if (FORM == 10) {
                    x[k] = mont32c(x[k], c, c * ninv, n);
                } else if (FORM == 11) {
                    // p = 2^31 - 1, b = c mod p, w = floor(b 2^32 / p); x < p
                    const uint32_t p = 2147483647u, b = c % p;
                    const uint32_t w = (uint32_t)(((uint64_t)b << 32) / p);
                    const uint32_t xx = x[k] & 0x7FFFFFFFu;
                    const uint32_t q = umulhi32(xx, w);
                    uint32_t r = xx * b - q * p;
                    x[k] = r >= p ? r - p : r;
                } else if (FORM == 7) {
                    // c < 2^31 <= n - 1; the result's low bits feed the next c
                    const double R = real32_fast(x[k] & 0x7FFFFFFFu, yN, ybits, W);
                    x[k] ^= (uint32_t)__double_as_longlong(R);
                } else {
                    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[k]) : "d"(0.999999), "d"(1e-7));
                }
            }
        }
    }
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) v ^= x[k] ^ (uint32_t)(acc[k] >> 32) ^ (uint32_t)(d[k] * 7.0);
    sink[tid] = v;
}

template <int FORM>
static int run_one(double *ops_per_s, cudaStream_t s, std::string *err)
{
    int dev = 0, sms = 0, blocks_per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, microbench_kernel<FORM>, 256, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const uint64_t grid = (uint64_t)sms * blocks_per_sm;
    uint32_t *sink = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&sink, grid * 256 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        *err = "microbench: allocation failed";
        return PHPRNG_ENOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // n = 2^32 - 5 (prime), its inverse mod 2^32
    const uint32_t n = 4294967291u;
    uint32_t ninv = n;
    for (int i = 0; i < 5; ++i) ninv *= 2u - n * ninv;
    int iters = FORM == 4 ? 64 : (FORM == 6 || FORM == 7) ? 16 : 256;
    // R of form 7 for n = 2^32 - 5, from the host's own derivation
    const phprng_instance in = {n, 3, 2147483647u, 784588716u, 0, 1};
    ExpProg pg;
    const DevInst P = derive_inst(in, 0, &pg);
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {            // warm-up, then two timed sizes
        cudaEventRecord(e0, s);
        microbench_kernel<FORM><<<(unsigned)grid, 256, 0, s>>>(sink, iters, 2654435769u, n, ninv, P.yN,
                                                               P.ybits, P.aux);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < 20.f && rep < 2) iters *= 4;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) {
        *err = std::string("microbench: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    const double ops = (double)grid * 256.0 * iters * kUnroll * kChains;
    *ops_per_s = ops / (ms * 1e-3);
    return PHPRNG_OK;
}

// Form 5: each warp runs its instance's program on 8 messages per lane and
// feeds the results back as the next messages (so no exponentiation can be
// skipped); the XOR of all results goes to sink only if it hits a constant.
__global__ void __launch_bounds__(256, 2) exp_kernel(const DevInst *inst, const ExpProg *prog,
                                                     int reps, uint32_t *sink)
{
    constexpr int NPT = 8;
    const int lane = threadIdx.x & 31;
    const uint64_t w = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const DevInst P = inst[w];
    const ExpProg &pg = prog[w];
    const uint32_t n = (uint32_t)P.n;
    uint32_t msg[NPT], x[NPT], acc = 0;
#pragma unroll
    for (int u = 0; u < NPT; ++u) msg[u] = (uint32_t)((w * 977 + lane * 131 + u * 7919) % n);
    for (int r = 0; r < reps; ++r) {
        modexp_prog<NPT, uint32_t>(x, msg, pg, n, (uint32_t)P.ninv, (uint32_t)P.K,
                                   (uint32_t)(P.ninv >> 32));
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            msg[u] = x[u];
            acc ^= x[u];
        }
    }
    if (acc == 0x9E3779B9u) sink[w * 32 + lane] = acc;
}

static int run_exp(double *ops_per_s, cudaStream_t s, std::string *err)
{
    const uint64_t count = 65536;
    const int reps = 16;
    std::vector<phprng_instance> in(count);
    int rc = draw_instances(32, count, 0x5EED0001, PHPRNG_REQUIRE_SAFE_PRIME, in.data(), err);
    if (rc != PHPRNG_OK) return rc;
    std::vector<DevInst> di(count);
    std::vector<ExpProg> pg(count);
    double products = 0;
    for (uint64_t i = 0; i < count; ++i) {
        di[i] = derive_inst(in[i], 0, &pg[i]);
        products += program_products(pg[i]);
    }
    DevInst *d_i = nullptr;
    ExpProg *d_p = nullptr;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t e = cudaMalloc(&d_i, count * sizeof(DevInst));
    if (e == cudaSuccess) e = cudaMalloc(&d_p, count * sizeof(ExpProg));
    if (e == cudaSuccess) e = cudaMalloc(&sink, count * 32 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_i, di.data(), count * sizeof(DevInst), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_p, pg.data(), count * sizeof(ExpProg), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {     // two warm-ups, one timed
        cudaEventRecord(e0, s);
        exp_kernel<<<(unsigned)(count / 8), 256, 0, s>>>(d_i, d_p, reps, sink);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_i);
    cudaFree(d_p);
    cudaFree(sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("microbench (exponentiation): ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? PHPRNG_ENOMEM : PHPRNG_ECUDA;
    }
    *ops_per_s = products * 32.0 * 8.0 * reps / (ms * 1e-3);
    return PHPRNG_OK;
}

int run_microbench(int which, double *ops_per_s, void *stream, std::string *err)
{
    cudaStream_t s = (cudaStream_t)stream;
    switch (which) {
    case 0: return run_one<0>(ops_per_s, s, err);
    case 1: return run_one<1>(ops_per_s, s, err);
    case 2: return run_one<2>(ops_per_s, s, err);
    case 3: return run_one<3>(ops_per_s, s, err);
    case 4: return run_one<4>(ops_per_s, s, err);
    case 5: return run_exp(ops_per_s, s, err);
    case 6: return run_one<6>(ops_per_s, s, err);
    case 7: return run_one<7>(ops_per_s, s, err);
    case 8: return run_one<8>(ops_per_s, s, err);
    case 9: return run_one<9>(ops_per_s, s, err);
    case 10: return run_one<10>(ops_per_s, s, err);
    case 11: return run_one<11>(ops_per_s, s, err);
    default:
        *err = "microbench: unknown form";
        return PHPRNG_EINVAL;
    }
}

}  // namespace phprng
