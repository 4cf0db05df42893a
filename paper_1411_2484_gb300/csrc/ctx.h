// ctx.h -- the context object behind the opaque phprng_ctx handle, shared by
// the C ABI (capi.cpp) and the serving loop (serve.cpp).
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

#define PH_API extern "C" __attribute__((visibility("default")))

using phprng::DevInst;
using phprng::DevState;
using phprng::ExpProg;
using phprng::ExpProg8;
using phprng::SkipConst;
using phprng::SkipTable;

struct phprng_ctx {
    int width = 32;
    uint64_t count = 0;
    uint32_t flags = 0;
    int device = 0;
    uint64_t p = 0, a = 0;
    bool any32 = false, any64 = false;
    std::vector<phprng_instance> host_inst;
    std::vector<uint8_t> wide;
    DevInst *d_inst = nullptr;
    ExpProg *d_prog = nullptr;        // exponent programs, one per instance
    ExpProg8 *d_prog8 = nullptr;      // the 32-bit kernels' exact-search programs, one per instance
    uint64_t *d_state = nullptr;      // 4 * count: m | s | c | pos
    DevState st{};
    SkipConst sk32{}, sk64{}, sk32_8{}, sk32_4{};
    std::vector<uint64_t> pos_host;   // host mirror of the stream positions
    // launch order: key[i] = 256*wide + 255 - products of instance i's program
    // (clamped; the exact-search program for 32-bit instances, which the
    // plain and test kernels run); key_std[i] the same by the standard
    // program, which the statistics kernel runs.  d_order[first ..] holds the
    // order of the last range sorted (indices relative to its first
    // instance), ord_first/ord_num name it.
    std::vector<uint16_t> key, key_std;
    uint32_t *d_order = nullptr;
    uint64_t ord_first = 0, ord_num = 0;
    // light-program decision of the last range launched (see launch_range)
    uint64_t lt_first = UINT64_MAX, lt_num = 0;
    bool lt_light = false;
    // skip-ahead: cycle positions of the seeds and the prefix table (lazy)
    uint64_t *d_L0 = nullptr, *d_m0 = nullptr, *d_T = nullptr;
    uint32_t *d_P = nullptr;
    SkipTable tbl{};
    bool skip_ready = false;
    // host-output staging: kStages device buffers, each with its own copy stream
    static constexpr int kStages = 3;
    void *stage[kStages] = {};
    size_t stage_bytes = 0;
    cudaStream_t copy_stream[kStages] = {};
    cudaEvent_t ev_done[kStages] = {}, ev_copied[kStages] = {};
    bool serving = false;             // a phprng_server owns the context
    // a wide skip prime (p >= 2^32, 64-bit moduli): skips are stepped in
    // 64-bit Montgomery arithmetic, skip-ahead sums formed by parallel
    // stepping (no prefix table), no split launches, no batched offsets
    bool wide_skip = false;
    phprng::SkipConst64 skw64{};
    uint64_t ainvM = 0;               // a^-1 2^64 mod p (going back)
    std::string err;
    std::mutex mu;
};


// Records the message for phprng_last_error and returns code.
int fail(phprng_ctx *ctx, int code, const std::string &msg);
int cuda_fail(phprng_ctx *ctx, cudaError_t e, const char *what);
// Builds the seeds' cycle positions and the skip prefix table once.
int ensure_skip(phprng_ctx *c, cudaStream_t s);

#define CU(ctx, call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);      \
    } while (0)
