// batch.cu -- batched persistent launch: many instances' requests of uneven
// lengths, at arbitrary stream positions, 32-bit and 64-bit moduli mixed, in
// one grid that stays resident and pulls tiles from a queue.
//
// A request (instance, start position, length) is cut on the host into tiles
// of at most `tile` numbers; tiles are sorted heaviest first (64-bit, then
// long) so the queue drains evenly.  Each warp of the persistent grid takes
// the next tile index with one atomic add and:
//   1. derives the state at the tile's start position from the instance's
//      seed (m0, s0 = a^L0) by Eq. 7 with the prefix table (skipdev.cuh) --
//      so tiles are independent of one another and of the stored state;
//   2. runs the tile's numbers exactly as the plain kernels do (gencore.cuh);
//   3. if the tile ends the last request of its instance, writes the state
//      back, so the context continues from there.
#include <cuda_runtime.h>

#include "gencore.cuh"
#include "skipdev.cuh"

namespace phprng {

#ifndef PH_BATCH_MINB
#define PH_BATCH_MINB 3
#endif

// Per warp: the exponent program's table, rows of 16 bytes per lane (32-bit
// tiles: up to kProg8MaxTable entries of NPT32/4 rows; 64-bit tiles: 4 entries
// of PH_NPT64/2 rows), in dynamic shared memory.
template <int NPT32>
struct BatchEtb {
    static constexpr int rows = kProg8MaxTable * (NPT32 / 4) > 4 * (PH_NPT64 / 2) ? kProg8MaxTable * (NPT32 / 4)
                                                                                   : 4 * (PH_NPT64 / 2);
    static constexpr size_t bytes = (size_t)8 * rows * 32 * sizeof(uint4);    // 8 warps per block
};
extern __shared__ uint4 g_batch_etb[];

template <int NPT, typename CT>
__device__ __forceinline__ void run_tile32(const BatchArgs &a, const DevInst &P, const ExpProg &pg,
                                           const ExpProg8 &pg8, uint64_t i, int lane, uint32_t m, uint32_t s,
                                           const Tile &T, bool wb, bool vec_ok, uint4 *etb)
{
    constexpr uint64_t G = 32 * NPT;
    const SkipConst &sk = NPT == 8 ? a.sk32_8 : a.sk32_4;
    uint32_t M = m;
    uint32_t sig = mont32(s, sk.lane[lane], sk.p, sk.pinv);
    CT *cdst = a.c_base ? (CT *)a.c_base + T.c_off : nullptr;
    double *rdst = a.r_base ? a.r_base + T.r_off : nullptr;
    const uint64_t len = T.len;
    uint32_t x[NPT], sig_last = sig;
    uint64_t g_last = 0;
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        uint32_t sv[NPT], msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        messages32<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
        encrypt32_p8<NPT>(P, pg, pg8, msg, x, etb, lane);
        store_group<NPT, CT, uint32_t>(P, cdst, rdst, my0, len, vec_ok, x);
    }
    if (wb) write_state_after<NPT, uint32_t, uint32_t>(a.st, sk, i, lane, g_last, len, T.start + len, M,
                                                       sig_last, x);
}

template <int NPT>
__device__ __forceinline__ void run_tile64(const BatchArgs &a, const DevInst &P, const ExpProg &pg,
                                           uint64_t i, int lane, uint64_t m, uint32_t s,
                                           const Tile &T, bool wb, bool vec_ok, uint4 *etb)
{
    constexpr uint64_t G = 32 * NPT;
    const SkipConst &sk = a.sk64;
    uint64_t M = m;
    uint32_t sig = mont32(s, sk.lane[lane], sk.p, sk.pinv);
    uint64_t *cdst = a.c_base ? (uint64_t *)a.c_base + T.c_off : nullptr;
    double *rdst = a.r_base ? a.r_base + T.r_off : nullptr;
    const uint64_t len = T.len;
    uint64_t x[NPT];
    uint32_t sig_last = sig;
    uint64_t g_last = 0;
    for (uint64_t g0 = 0; g0 < len; g0 += G) {
        uint32_t sv[NPT];
        uint64_t msg[NPT];
        const uint64_t my0 = g0 + (uint64_t)NPT * lane;
        sig_last = sig;
        g_last = g0;
        messages64<NPT>(P, sk, lane, my0, len, M, sig, sv, msg);
        encrypt_tb<NPT, uint64_t>(P, pg, msg, x, etb, lane);
        store_group<NPT, uint64_t, uint64_t>(P, cdst, rdst, my0, len, vec_ok, x);
    }
    if (wb) write_state_after<NPT, uint64_t, uint64_t>(a.st, sk, i, lane, g_last, len, T.start + len, M,
                                                       sig_last, x);
}

template <int NPT32, typename CT>
__global__ void __launch_bounds__(256, PH_BATCH_MINB) batch_kernel(BatchArgs a)
{
    const int lane = threadIdx.x & 31;
    uint4 *etb = g_batch_etb + (threadIdx.x >> 5) * BatchEtb<NPT32>::rows * 32;   // this warp's table
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1ull);
        t = __shfl_sync(kFullMask, t, 0);
        if (t >= a.ntiles) return;
        const Tile T = a.tiles[t];
        const uint64_t i = T.inst & kTileInstMask;
        const bool wide = (T.inst & kTileWide) != 0, wb = (T.inst & kTileWriteBack) != 0;
        const DevInst P = a.inst[i];
        uint64_t m, L;
        uint32_t s;
        skip_state_warp(a.tb, P, a.m0[i], a.L0[i], T.start, &m, &s, &L);   // Eq. 7
        const bool vec_ok = a.vec_ok && (T.c_off % (16 / sizeof(CT)) == 0) && (T.r_off % 2 == 0);
        if (!wide)
            run_tile32<NPT32, CT>(a, P, a.prog[i], a.prog8[i], i, lane, (uint32_t)m, s, T, wb, vec_ok, etb);
        else
            run_tile64<PH_NPT64>(a, P, a.prog[i], i, lane, m, s, T, wb,
                          a.vec_ok && (T.c_off % 2 == 0) && (T.r_off % 2 == 0), etb);
    }
}

// The launch's dynamic shared memory; above the default 48 KiB the kernel's
// limit is raised first (current device), as the occupancy query needs too.
template <int NPT32, typename CT>
static size_t batch_smem()
{
    constexpr size_t smem = BatchEtb<NPT32>::bytes;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(batch_kernel<NPT32, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return smem;
}

template <int NPT32, typename CT>
static int launch_one(const BatchArgs &a, int blocks_per_sm, void *stream, std::string *err)
{
    int dev = 0, sms = 0, maxb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = batch_smem<NPT32, CT>();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_kernel<NPT32, CT>, 256, smem);
    if (maxb < 1) maxb = 1;
    const int b = blocks_per_sm <= 0 || blocks_per_sm > maxb ? maxb : blocks_per_sm;
    uint64_t grid = (uint64_t)sms * b;
    const uint64_t warps_needed = (a.ntiles + 7) / 8;
    if (grid > warps_needed) grid = warps_needed ? warps_needed : 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        *err = std::string("batch counter reset: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    batch_kernel<NPT32, CT><<<(unsigned)grid, 256, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("batch_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_batch(const BatchArgs &a, int npt32, int blocks_per_sm, void *stream, std::string *err)
{
    if (a.ntiles == 0) return PHPRNG_OK;
    if (a.c_is_64)
        return npt32 == 4 ? launch_one<4, uint64_t>(a, blocks_per_sm, stream, err)
                          : launch_one<8, uint64_t>(a, blocks_per_sm, stream, err);
    return npt32 == 4 ? launch_one<4, uint32_t>(a, blocks_per_sm, stream, err)
                      : launch_one<8, uint32_t>(a, blocks_per_sm, stream, err);
}

int batch_max_blocks_per_sm(int npt32, int c_is_64)
{
    int maxb = 0;
    if (c_is_64) {
        if (npt32 == 4)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_kernel<4, uint64_t>, 256,
                                                          batch_smem<4, uint64_t>());
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_kernel<8, uint64_t>, 256,
                                                          batch_smem<8, uint64_t>());
    } else {
        if (npt32 == 4)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_kernel<4, uint32_t>, 256,
                                                          batch_smem<4, uint32_t>());
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_kernel<8, uint32_t>, 256,
                                                          batch_smem<8, uint32_t>());
    }
    return maxb;
}

}  // namespace phprng
