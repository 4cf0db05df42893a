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
#include <cuda_runtime.h>

#include "arith.cuh"
#include "internal.h"

namespace phprng {

static constexpr int kChains = 8, kUnroll = 16;

template <int FORM>
__global__ void __launch_bounds__(256) microbench_kernel(uint32_t *sink, int iters, uint32_t c,
                                                         uint32_t n, uint32_t ninv)
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
    int iters = FORM == 4 ? 64 : 256;
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {            // warm-up, then two timed sizes
        cudaEventRecord(e0, s);
        microbench_kernel<FORM><<<(unsigned)grid, 256, 0, s>>>(sink, iters, 2654435769u, n, ninv);
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

int run_microbench(int which, double *ops_per_s, void *stream, std::string *err)
{
    cudaStream_t s = (cudaStream_t)stream;
    switch (which) {
    case 0: return run_one<0>(ops_per_s, s, err);
    case 1: return run_one<1>(ops_per_s, s, err);
    case 2: return run_one<2>(ops_per_s, s, err);
    case 3: return run_one<3>(ops_per_s, s, err);
    case 4: return run_one<4>(ops_per_s, s, err);
    default:
        *err = "microbench: unknown form";
        return PHPRNG_EINVAL;
    }
}

}  // namespace phprng
