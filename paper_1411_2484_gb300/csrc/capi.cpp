// capi.cpp -- the C ABI declared in include/phprng.h.
//
// A context owns, in device memory: the instance table (DevInst, 64 B per
// instance), the generator state (m, s, c, pos as four arrays of uint64) and,
// once a skip is requested, the prefix table of the skip cycle.  It also owns
// two staging buffers and a copy stream used only when a caller passes host
// output pointers.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cstring>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"

using namespace phprng;

static thread_local std::string g_err;

int fail(phprng_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg; else g_err = msg;
    return code;
}

int cuda_fail(phprng_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, PHPRNG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static void free_ctx(phprng_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    cudaFree(c->d_inst);
    cudaFree(c->d_prog);
    cudaFree(c->d_prog8);
    cudaFree(c->d_state);
    cudaFree(c->d_order);
    cudaFree(c->d_L0);
    cudaFree(c->d_m0);
    cudaFree(c->d_T);
    cudaFree(c->d_P);
    for (int k = 0; k < phprng_ctx::kStages; ++k) {
        cudaFree(c->stage[k]);
        if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
        if (c->copy_stream[k]) cudaStreamDestroy(c->copy_stream[k]);
    }
    delete c;
}

PH_API const char *phprng_status_string(int s)
{
    switch (s) {
    case PHPRNG_OK: return "ok";
    case PHPRNG_EINVAL: return "invalid argument";
    case PHPRNG_ENOTPRIME: return "modulus is not prime";
    case PHPRNG_EEXPONENT: return "exponent not coprime to n-1 or out of range";
    case PHPRNG_ESKIP: return "invalid skip generator";
    case PHPRNG_EDUPLICATE: return "duplicate modulus";
    case PHPRNG_ENOMEM: return "out of memory";
    case PHPRNG_ECUDA: return "CUDA error";
    case PHPRNG_ETIMEOUT: return "timed out";
    case PHPRNG_EBUDGET: return "output budget exhausted";
    default: return "unknown status";
    }
}

PH_API const char *phprng_last_error(const phprng_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

PH_API int phprng_is_prime(uint64_t n) { return is_prime(n) ? 1 : 0; }

PH_API int phprng_validate(int width, const phprng_instance *inst, uint64_t count,
                           uint32_t flags, uint64_t *bad_index)
{
    std::string msg;
    int rc = validate_all(width, inst, count, flags, bad_index, &msg);
    if (rc != PHPRNG_OK) g_err = msg;
    return rc;
}

PH_API int phprng_draw_instances(int width, uint64_t count, uint64_t seed, uint32_t flags,
                                 phprng_instance *out)
{
    std::string msg;
    int rc;
    try {
        rc = draw_instances(width, count, seed, flags, out, &msg);
    } catch (const std::bad_alloc &) {
        msg = "phprng_draw_instances: host allocation failed";
        rc = PHPRNG_ENOMEM;
    }
    if (rc != PHPRNG_OK) g_err = msg;
    return rc;
}

// Launch order of instances first .. first+num-1: 32-bit instances before
// 64-bit ones, each heaviest program first, so that the warps of a block --
// which hold the block's resources until the slowest is done -- carry equal
// work, and the last wave holds the lightest blocks.  Below this many
// instances a launch is too short for the order to matter.
static constexpr uint64_t kOrderMinInstances = 1024;

// Device order for a range (indices relative to `first`), sorted on the host
// by a counting sort of the instances' keys and copied on stream s, or reused
// when the range is the one sorted last.  Calls on overlapping instance ranges
// must be ordered on the device anyway (they share stream states); the order
// of a range lives in the slots of its own instances.
static const uint32_t *instance_order(phprng_ctx *c, uint64_t first, uint64_t num,
                                      cudaStream_t s, int *rc)
{
    *rc = PHPRNG_OK;
    if (c->ord_num == num && c->ord_first == first) return c->d_order + first;
    std::vector<uint32_t> ord, cnt(513, 0);
    try {
        ord.resize(num);
    } catch (const std::bad_alloc &) {
        *rc = fail(c, PHPRNG_ENOMEM, "instance order: host allocation failed");
        return nullptr;
    }
    for (uint64_t j = 0; j < num; ++j) ++cnt[c->key[first + j] + 1];
    for (int k = 1; k <= 512; ++k) cnt[k] += cnt[k - 1];
    for (uint64_t j = 0; j < num; ++j) ord[cnt[c->key[first + j]]++] = (uint32_t)j;
    // from pageable memory: staged before the call returns, then ordered on s
    cudaError_t e = cudaMemcpyAsync(c->d_order + first, ord.data(), num * sizeof(uint32_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        *rc = cuda_fail(c, e, "instance order upload");
        return nullptr;
    }
    c->ord_first = first;
    c->ord_num = num;
    return c->d_order + first;
}

PH_API int phprng_create(phprng_ctx **out, int width, const phprng_instance *inst,
                         uint64_t count, uint32_t flags, void *cuda_stream)
{
    if (!out) return fail(nullptr, PHPRNG_EINVAL, "phprng_create: out is NULL");
    *out = nullptr;
    std::string msg;
    uint64_t bad = 0;
    int rc;
    try {
        rc = validate_all(width, inst, count, flags, &bad, &msg);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, PHPRNG_ENOMEM, "phprng_create: host allocation failed");
    }
    if (rc != PHPRNG_OK) return fail(nullptr, rc, "phprng_create: " + msg);

    phprng_ctx *c = new (std::nothrow) phprng_ctx;
    if (!c) return fail(nullptr, PHPRNG_ENOMEM, "phprng_create: host allocation failed");
    std::vector<DevInst> di;
    std::vector<ExpProg> prog;
    std::vector<ExpProg8> prog8;
    std::vector<uint64_t> state;
    try {
        c->width = width;
        c->count = count;
        c->flags = flags;
        c->p = inst[0].p;
        c->a = inst[0].a;
        c->host_inst.assign(inst, inst + count);
        c->pos_host.assign(count, 0);
        c->wide.resize(count);
        c->key.resize(count);
        c->key_std.resize(count);
        di.resize(count);
        prog.resize(count);
        prog8.resize(count);
        state.assign(4 * count, 0);
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(nullptr, PHPRNG_ENOMEM, "phprng_create: host allocation failed");
    }
    for (uint64_t i = 0; i < count; ++i) {
        int w = width == 64 ? 1 : width == 32 ? 0 : (inst[i].n >= (1ull << 32) ? 1 : 0);
        c->wide[i] = (uint8_t)w;
        (w ? c->any64 : c->any32) = true;
        di[i] = derive_inst(inst[i], w, &prog[i]);
        if (!w) prog8[i] = derive_prog8(inst[i].n, inst[i].e);   // the 32-bit kernels' program
        c->key[i] = (uint16_t)(256 * w + 255 - std::min(w ? program_products(prog[i]) : program8_products(prog8[i]), 255));
        c->key_std[i] = (uint16_t)(256 * w + 255 - std::min(program_products(prog[i]), 255));
        state[i] = inst[i].m0;
        state[count + i] = inst[i].s0;
    }
    if (c->p >= (1ull << 32)) {
        // the Implementation section's wide skip generator for 64-bit moduli
        c->wide_skip = true;
        c->skw64 = phprng::derive_skip64(c->p, c->a, gen_npt(1));
        const uint64_t R = (uint64_t)((((unsigned __int128)1) << 64) % c->p);
        c->ainvM = mulmod(powmod(c->a, c->p - 2, c->p), R, c->p);
    } else {
        c->sk32 = derive_skip(c->p, c->a, gen_npt(0));
        c->sk64 = derive_skip(c->p, c->a, gen_npt(1));
        c->sk32_8 = derive_skip(c->p, c->a, 8);
        c->sk32_4 = derive_skip(c->p, c->a, 4);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_inst, count * sizeof(DevInst));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_prog, count * sizeof(ExpProg));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_prog8, count * sizeof(ExpProg8));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_state, 4 * count * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_order, count * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_prog, prog.data(), count * sizeof(ExpProg), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_prog8, prog8.data(), count * sizeof(ExpProg8), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_inst, di.data(), count * sizeof(DevInst), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_state, state.data(), 4 * count * sizeof(uint64_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors die on return
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? PHPRNG_ENOMEM : PHPRNG_ECUDA;
        std::string m = std::string("phprng_create: ") + cudaGetErrorString(e);
        free_ctx(c);
        return fail(nullptr, code, m);
    }
    c->st.m = c->d_state;
    c->st.s = c->d_state + count;
    c->st.c = c->d_state + 2 * count;
    c->st.pos = c->d_state + 3 * count;
    if (count >= kOrderMinInstances) {               // the whole table's order, ready for use
        int orc = PHPRNG_OK;
        instance_order(c, 0, count, s, &orc);
        if (orc == PHPRNG_OK && cudaStreamSynchronize(s) != cudaSuccess) orc = PHPRNG_ECUDA;
        if (orc != PHPRNG_OK) {
            std::string m = "phprng_create: " + c->err;
            free_ctx(c);
            return fail(nullptr, orc, m);
        }
    }
    *out = c;
    return PHPRNG_OK;
}

PH_API int phprng_create_seeded(phprng_ctx **out, int width, uint64_t count, uint64_t seed,
                                uint32_t flags, void *cuda_stream)
{
    if (!out) return fail(nullptr, PHPRNG_EINVAL, "phprng_create_seeded: out is NULL");
    *out = nullptr;
    if (width != 32 && width != 64)
        return fail(nullptr, PHPRNG_EINVAL, "phprng_create_seeded: width must be 32 or 64");
    std::vector<phprng_instance> v;
    try {
        v.resize(count);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, PHPRNG_ENOMEM, "phprng_create_seeded: host allocation failed");
    }
    std::string msg;
    int rc = draw_instances(width, count, seed, flags, v.data(), &msg);
    if (rc != PHPRNG_OK) return fail(nullptr, rc, msg);
    return phprng_create(out, width, v.data(), count, flags, cuda_stream);
}

PH_API int phprng_destroy(phprng_ctx *ctx)
{
    if (ctx && ctx->serving)
        return fail(ctx, PHPRNG_EINVAL, "phprng_destroy: destroy the server first");
    free_ctx(ctx);
    return PHPRNG_OK;
}

// Kind of memory behind a pointer: 1 device (or managed), 0 host, -1 error.
static int pointer_kind(const void *p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return -1; }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

// Split launches (SplitArgs): a call with fewer instances than eight times
// the warps the GPU keeps resident may cut each instance into K chunks of Lc
// numbers (Lc a multiple of 256, at least kMinChunk; K at most kMaxSplit) so
// the grid fills the GPU.  K is chosen to minimise the estimated time
// waves * (Lc + kChunkCost) over 1 to 64 waves: waves = ceil(num K / resident
// warps), kChunkCost
// the per-chunk start (its skip power, its start message and its share of the
// pre-pass) in numbers; K = 1 when no split beats the unsplit launch.  The
// chunk starts cost one extra skip product per number (the pre-pass) and a
// short sum per warp.
static constexpr uint32_t kMaxSplit = 4096;
#ifndef PH_MIN_CHUNK
#define PH_MIN_CHUNK 1024
#endif
static constexpr uint64_t kMinChunk = PH_MIN_CHUNK;
static constexpr uint64_t kChunkCost = 128;

// The chunk count of a split launch (1: none) for num instances of per_inst
// numbers with `resident` warps resident on the GPU; *Lc the chunk length.
static uint32_t split_chunks(uint64_t num, uint64_t per_inst, uint64_t resident, uint64_t *Lc)
{
    *Lc = per_inst;
    if (num == 0 || resident == 0 || num >= 8 * resident || per_inst < 2 * kMinChunk) return 1;
    uint64_t best_cost = (num + resident - 1) / resident * (per_inst + kChunkCost);
    uint32_t best = 1;
    // for each wave count w the cheapest split is the shortest chunk that keeps
    // num * K within w waves
    for (uint64_t w = 1; w <= 64; ++w) {
        const uint64_t Kmax = std::min<uint64_t>(w * resident / num, kMaxSplit);
        if (Kmax < 2) continue;
        const uint64_t L = std::max<uint64_t>(((per_inst + Kmax - 1) / Kmax + 255) / 256 * 256,
                                              (kMinChunk + 255) / 256 * 256);
        const uint64_t K = (per_inst + L - 1) / L;      // chunks in use (none empty)
        if (K < 2 || K > kMaxSplit) continue;
        const uint64_t cost = (num * K + resident - 1) / resident * (L + kChunkCost);
        if (cost < best_cost) {
            best_cost = cost;
            best = (uint32_t)K;
            *Lc = L;
        }
    }
    return best;
}

static int prepare_split(phprng_ctx *c, uint64_t num, uint64_t per_inst, GenArgs *g, cudaStream_t s)
{
    if (c->wide_skip) return PHPRNG_OK;               // wide skips: never split
    uint64_t Lc = 0;
    const uint32_t K = split_chunks(num, per_inst, gen_resident_warps(), &Lc);
    if (K == 1) return PHPRNG_OK;
    SplitArgs &sp = g->sp;
    sp.K = K;
    sp.Kinv = (uint64_t)((((unsigned __int128)1 << 64) + K - 1) / K);
    sp.Lc = Lc;
    const uint64_t pm = c->sk32_8.p;                 // the skip products' modulus (3 for the unit skip)
    const uint64_t R = (1ull << 32) % pm;
    sp.oneM = (uint32_t)R;
    sp.aLcM = (uint32_t)mulmod(powmod(c->a, sp.Lc, pm), R, pm);
    uint64_t *scr = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&scr, num * (K + 1) * sizeof(uint64_t), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sp = SplitArgs();
        return fail(c, PHPRNG_ENOMEM, "phprng_generate: split scratch allocation failed");
    }
    sp.scratch = scr;
    std::string err;
    int rc = launch_chunk_sums(*g, c->sk32_8, s, &err);
    if (rc != PHPRNG_OK) {
        cudaFreeAsync(scr, s);
        sp = SplitArgs();
        return fail(c, rc, "phprng_generate: " + err);
    }
    return PHPRNG_OK;
}

// Launches whose 32-bit instances average at most this many Montgomery
// products per exponentiation (the paper's small exponents: 3 to 6) run the
// generator's LIGHT instantiation.
static constexpr double kLightProducts = 12.0;

static bool light_range(phprng_ctx *c, uint64_t first, uint64_t num)
{
    if (c->lt_first == first && c->lt_num == num) return c->lt_light;
    uint64_t sum = 0, cnt = 0;
    for (uint64_t j = first; j < first + num; ++j) {
        if (c->key_std[j] >= 256) continue;              // 64-bit instance
        sum += 255 - c->key_std[j];                      // the LIGHT loop runs the standard program
        ++cnt;
    }
    c->lt_first = first;
    c->lt_num = num;
    c->lt_light = cnt && (double)sum / (double)cnt <= kLightProducts;
    return c->lt_light;
}

static int launch_range(phprng_ctx *c, uint64_t first, uint64_t num, uint64_t per_inst,
                        void *c_out, double *r_out, phprng_stats *stats, cudaStream_t s,
                        bool ordered = false)
{
    GenArgs g;
    if (ordered && !stats && num >= kOrderMinInstances && num < (1ull << 32)) {
        int rc = PHPRNG_OK;
        g.order = instance_order(c, first, num, s, &rc);
        if (rc != PHPRNG_OK) return rc;
    }
    g.inst = c->d_inst;
    g.prog = c->d_prog;
    g.prog8 = c->d_prog8;
    g.st = c->st;
    g.first = first;
    g.num = num;
    g.per_inst = per_inst;
    g.c_out = c_out;
    g.r_out = r_out;
    g.stats = stats;
    g.edge = nullptr;
    g.c_is_64 = c->width != 32;
    const size_t csz = g.c_is_64 ? 8 : 4;
    g.vec_ok = (per_inst % 4 == 0) && ((uintptr_t)c_out % 16 == 0) &&
               ((uintptr_t)r_out % 16 == 0) && (csz * per_inst) % 16 == 0;
    std::string err;
    int rc = PHPRNG_OK;
    if (!stats) {
        rc = prepare_split(c, num, per_inst, &g, s);
        if (rc != PHPRNG_OK) return rc;
    }
    const uint64_t edge_words = stats ? gen32_edge_words(num, per_inst) : 0;
    if (edge_words) {
        cudaError_t e = cudaMallocAsync((void **)&g.edge, edge_words * 4, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PHPRNG_ENOMEM, "phprng_generate: statistics scratch allocation failed");
        }
    }
    // statistics: blocks of consecutive instances (their adjacent-stream
    // products need them together), launched heaviest block first
    uint32_t *bord = nullptr;
    if (stats && num >= kOrderMinInstances && num < (1ull << 32)) {
        const uint64_t W = gen32_stats_block_warps(), nb = (num + W - 1) / W;
        std::vector<uint32_t> ord(nb), cnt(513, 0);
        auto bkey = [&](uint64_t b) {
            uint16_t k = c->key_std[first + W * b];
            for (uint64_t j = W * b + 1; j < std::min<uint64_t>(num, W * b + W); ++j)
                k = std::min(k, c->key_std[first + j]);
            return k;
        };
        for (uint64_t b = 0; b < nb; ++b) ++cnt[bkey(b) + 1];
        for (int k = 1; k <= 512; ++k) cnt[k] += cnt[k - 1];
        for (uint64_t b = 0; b < nb; ++b) ord[cnt[bkey(b)]++] = (uint32_t)b;
        // from pageable memory: staged before the call returns
        cudaError_t e = cudaMallocAsync((void **)&bord, nb * sizeof(uint32_t), s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bord, ord.data(), nb * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (bord) cudaFreeAsync(bord, s);
            if (g.edge) cudaFreeAsync(g.edge, s);
            return fail(c, PHPRNG_ENOMEM, "phprng_generate: statistics block order upload failed");
        }
        g.order = bord;
    }
    if (c->any32) {
        g.sk = c->sk32;
        g.light = !stats && light_range(c, first, num);
        rc = launch_gen32(g, s, &err);
    }
    if (bord) cudaFreeAsync(bord, s);
    if (g.edge) cudaFreeAsync(g.edge, s);
    if (rc == PHPRNG_OK && c->any64) {
        g.sk = c->sk64;
        g.wide_skip = c->wide_skip ? 1 : 0;
        g.skw = c->skw64;
        rc = launch_gen64(g, s, &err);
    }
    if (g.sp.scratch) cudaFreeAsync((void *)g.sp.scratch, s);
    if (rc != PHPRNG_OK) return fail(c, rc, "phprng_generate: " + err);
    return PHPRNG_OK;
}

static int ensure_staging(phprng_ctx *c, size_t bytes)
{
    const int S = phprng_ctx::kStages;
    if (c->stage_bytes >= bytes) return PHPRNG_OK;
    for (int k = 0; k < S; ++k) {
        cudaFree(c->stage[k]);
        c->stage[k] = nullptr;
    }
    c->stage_bytes = 0;
    for (int k = 0; k < S; ++k) {
        cudaError_t e = cudaMalloc(&c->stage[k], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PHPRNG_ENOMEM, "phprng_generate: staging allocation failed");
        }
        if (!c->ev_done[k]) CU(c, cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming));
        if (!c->ev_copied[k]) CU(c, cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
        if (!c->copy_stream[k])
            CU(c, cudaStreamCreateWithFlags(&c->copy_stream[k], cudaStreamNonBlocking));
    }
    c->stage_bytes = bytes;
    return PHPRNG_OK;
}

// Host outputs: generate blocks (instances x numbers) into kStages device
// staging buffers in turn and copy each block back on that buffer's own copy
// stream while later blocks are generated (several copy engines can run at
// once); every block is one contiguous copy.  The first block of whole
// instances is kept to about 2^22 numbers, so that the first copy starts
// early.  Returns once everything is on the host.
static int generate_to_host(phprng_ctx *c, uint64_t first, uint64_t num, uint64_t per_inst,
                            void *c_out, double *r_out, cudaStream_t s)
{
    const int S = phprng_ctx::kStages;
    const size_t csz = c->width == 32 ? 4 : 8;
    const size_t per_num = (c_out ? csz : 0) + (r_out ? 8 : 0);
    const uint64_t cap = 1ull << 25;                      // numbers per block
    const uint64_t piece = std::min<uint64_t>(per_inst, cap);
    const uint64_t ninst = std::max<uint64_t>(1, std::min<uint64_t>(num, cap / piece));
    int rc = ensure_staging(c, (size_t)(ninst * piece * per_num + 256));
    if (rc != PHPRNG_OK) return rc;
    int k = 0;
    bool used[phprng_ctx::kStages] = {};
    const uint64_t ninst0 = std::max<uint64_t>(1, std::min<uint64_t>(ninst, (1ull << 22) / piece));
    for (uint64_t i0 = 0, ni = 0; i0 < num; i0 += ni) {
        ni = std::min(i0 == 0 ? ninst0 : ninst, num - i0);
        for (uint64_t j0 = 0; j0 < per_inst; j0 += piece) {
            const uint64_t pj = std::min(piece, per_inst - j0);
            char *buf = (char *)c->stage[k];
            void *dc = c_out ? buf : nullptr;
            double *dr = r_out ? (double *)(buf + ((c_out ? ni * pj * csz : 0) + 15) / 16 * 16)
                               : nullptr;
            if (used[k]) CU(c, cudaStreamWaitEvent(s, c->ev_copied[k], 0));
            rc = launch_range(c, first + i0, ni, pj, dc, dr, nullptr, s);
            if (rc != PHPRNG_OK) return rc;
            CU(c, cudaEventRecord(c->ev_done[k], s));
            cudaStream_t cs = c->copy_stream[k];
            CU(c, cudaStreamWaitEvent(cs, c->ev_done[k], 0));
            // A block is either whole instances (pj == per_inst) or a piece of a
            // single instance (ni == 1), so its host image is one contiguous run.
            if (c_out)
                CU(c, cudaMemcpyAsync((char *)c_out + (i0 * per_inst + j0) * csz, dc, ni * pj * csz,
                                      cudaMemcpyDeviceToHost, cs));
            if (r_out)
                CU(c, cudaMemcpyAsync(r_out + i0 * per_inst + j0, dr, ni * pj * 8,
                                      cudaMemcpyDeviceToHost, cs));
            CU(c, cudaEventRecord(c->ev_copied[k], cs));
            used[k] = true;
            k = (k + 1) % S;
        }
    }
    for (int j = 0; j < S; ++j)
        if (used[j]) CU(c, cudaStreamSynchronize(c->copy_stream[j]));
    CU(c, cudaStreamSynchronize(s));
    return PHPRNG_OK;
}

PH_API int phprng_generate(phprng_ctx *ctx, uint64_t first, uint64_t num_inst,
                           uint64_t per_inst, void *c_out, double *r_out,
                           phprng_stats *stats_out, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_generate: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_generate: a server owns the context");
    if (first > ctx->count || num_inst > ctx->count - first)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate: instance range outside the table");
    if (num_inst == 0 || per_inst == 0) return PHPRNG_OK;
    if (num_inst > (1ull << 40) / per_inst)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate: num_inst * per_inst exceeds 2^40");
    const size_t csz = ctx->width == 32 ? 4 : 8;
    if (((uintptr_t)c_out % csz) || ((uintptr_t)r_out % 8))
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate: output pointer not aligned to its element");
    if (stats_out) {
        if (ctx->any64)
            return fail(ctx, PHPRNG_EINVAL,
                        "phprng_generate: fused statistics are defined for 32-bit moduli only");
        if (per_inst >= (1ull << 31))
            return fail(ctx, PHPRNG_EINVAL, "phprng_generate: statistics need per_inst < 2^31");
        if ((uintptr_t)stats_out % 8)
            return fail(ctx, PHPRNG_EINVAL, "phprng_generate: stats_out not 8-byte aligned");
    }
    if (!c_out && !r_out && !stats_out)
        return fail(ctx, PHPRNG_EINVAL,
                    "phprng_generate: no output (use phprng_skip to advance without output)");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const int kc = c_out ? pointer_kind(c_out) : -2;
    const int kr = r_out ? pointer_kind(r_out) : -2;
    if (kc == -1 || kr == -1)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate: cannot classify an output pointer");
    const bool host = (kc == 0) || (kr == 0);
    const bool dev = (kc == 1) || (kr == 1);
    if (host && dev)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate: mix of host and device output pointers");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc;
    if (stats_out) {
        if (host)
            return fail(ctx, PHPRNG_EINVAL,
                        "phprng_generate: with statistics, c_out/r_out must be device memory");
        const int ks = pointer_kind(stats_out);
        if (ks == -1)
            return fail(ctx, PHPRNG_EINVAL, "phprng_generate: cannot classify stats_out");
        if (ks == 1) {
            rc = launch_range(ctx, first, num_inst, per_inst, c_out, r_out, stats_out, s);
        } else {                                 // host statistics: stage, copy back, wait
            phprng_stats *d = nullptr;
            CU(ctx, cudaMallocAsync((void **)&d, num_inst * sizeof(phprng_stats), s));
            rc = launch_range(ctx, first, num_inst, per_inst, c_out, r_out, d, s);
            cudaError_t e = rc == PHPRNG_OK
                ? cudaMemcpyAsync(stats_out, d, num_inst * sizeof(phprng_stats),
                                  cudaMemcpyDeviceToHost, s)
                : cudaSuccess;
            cudaFreeAsync(d, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (rc == PHPRNG_OK && e != cudaSuccess) return cuda_fail(ctx, e, "phprng_generate: statistics copy");
        }
    } else {
        // Host outputs, pinned or not, go through device staging: the copy
        // engines move them at about 4.5 times the rate of kernel stores into
        // mapped pinned memory (183 vs 41 GB/s measured on GB300).
        rc = host ? generate_to_host(ctx, first, num_inst, per_inst, c_out, r_out, s)
                  : launch_range(ctx, first, num_inst, per_inst, c_out, r_out, nullptr, s, true);
    }
    if (rc == PHPRNG_OK)
        for (uint64_t i = first; i < first + num_inst; ++i) ctx->pos_host[i] += per_inst;
    return rc;
}

PH_API int phprng_generate_stats_noalloc(phprng_ctx *ctx, uint64_t first, uint64_t num_inst,
                                        uint64_t per_inst, phprng_stats *stats_out,
                                        void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_generate_stats_noalloc: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate_stats_noalloc: a server owns the context");
    if (first > ctx->count || num_inst > ctx->count - first)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate_stats_noalloc: instance range outside the table");
    if (ctx->any64)
        return fail(ctx, PHPRNG_EINVAL,
                    "phprng_generate_stats_noalloc: statistics are defined for 32-bit moduli only");
    if (per_inst >= (1ull << 31))
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate_stats_noalloc: per_inst must be below 2^31");
    if (num_inst == 0 || per_inst == 0) return PHPRNG_OK;
    if (!stats_out || (uintptr_t)stats_out % 8)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate_stats_noalloc: stats_out NULL or misaligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (pointer_kind(stats_out) != 1)
        return fail(ctx, PHPRNG_EINVAL, "phprng_generate_stats_noalloc: stats_out must be device memory");
    GenArgs g;
    g.inst = ctx->d_inst;
    g.prog = ctx->d_prog;
    g.prog8 = ctx->d_prog8;
    g.st = ctx->st;
    g.sk = ctx->sk32;
    g.first = first;
    g.num = num_inst;
    g.per_inst = per_inst;
    g.c_out = nullptr;
    g.r_out = nullptr;
    g.stats = stats_out;
    g.edge = nullptr;
    g.c_is_64 = ctx->width != 32;
    g.vec_ok = 1;
    std::string err;
    int rc = launch_gen32_stats_fixed(g, ctx->device, cuda_stream, &err);
    if (rc != PHPRNG_OK) return fail(ctx, rc, "phprng_generate_stats_noalloc: " + err);
    for (uint64_t i = first; i < first + num_inst; ++i) ctx->pos_host[i] += per_inst;
    return PHPRNG_OK;
}

PH_API int phprng_get_state(phprng_ctx *ctx, uint64_t inst, phprng_instance *state_out,
                            uint64_t *pos_out, uint64_t *c_out, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_get_state: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (inst >= ctx->count) return fail(ctx, PHPRNG_EINVAL, "phprng_get_state: instance out of range");
    if (!state_out) return fail(ctx, PHPRNG_EINVAL, "phprng_get_state: state_out is NULL");
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaStreamSynchronize((cudaStream_t)cuda_stream));
    uint64_t v[4];
    for (int k = 0; k < 4; ++k)
        CU(ctx, cudaMemcpy(&v[k], ctx->d_state + (uint64_t)k * ctx->count + inst, 8,
                           cudaMemcpyDeviceToHost));
    *state_out = ctx->host_inst[inst];
    state_out->m0 = v[0];
    state_out->s0 = v[1];
    if (c_out) *c_out = v[2];
    if (pos_out) *pos_out = v[3];
    return PHPRNG_OK;
}

// Builds, once per context, the cycle positions L0 of the seeds (discrete
// logs on the host) and the prefix table of the skip cycle (on the device).
int ensure_skip(phprng_ctx *c, cudaStream_t s)
{
    if (c->skip_ready) return PHPRNG_OK;
    std::vector<uint64_t> s0(c->count), L0(c->count), m0(c->count);
    for (uint64_t i = 0; i < c->count; ++i) {
        s0[i] = c->host_inst[i].s0;
        m0[i] = c->host_inst[i].m0;
    }
    SkipTable tb = derive_skip_table(c->p, c->a);
    if (tb.kind == 1) {
        // constant skip: the per-instance array holds the constant b = s0;
        // a skip is the closed form m + k b, so there is no table to build
        cudaError_t e = cudaMalloc(&c->d_L0, c->count * 8);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_m0, c->count * 8);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_L0, s0.data(), c->count * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_m0, m0.data(), c->count * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(c->d_L0); cudaFree(c->d_m0);
            c->d_L0 = c->d_m0 = nullptr;
            return cuda_fail(c, e, "phprng_skip: seed upload");
        }
        c->tbl = tb;
        c->skip_ready = true;
        return PHPRNG_OK;
    }
    if (!discrete_logs(c->p, c->a, s0.data(), c->count, L0.data()))
        return fail(c, PHPRNG_ESKIP, "phprng_skip: no discrete log for a seed s0 (a not a primitive root?)");
    uint64_t *seg = nullptr;
    cudaError_t e = cudaMalloc(&c->d_L0, c->count * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_m0, c->count * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_T, tb.nT * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_P, tb.nT * 4);
    if (e == cudaSuccess) e = cudaMalloc(&seg, tb.nT * 8);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_L0, L0.data(), c->count * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_m0, m0.data(), c->count * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaFree(seg);
        cudaFree(c->d_L0); cudaFree(c->d_m0); cudaFree(c->d_T); cudaFree(c->d_P);
        c->d_L0 = c->d_m0 = c->d_T = nullptr; c->d_P = nullptr;
        return cuda_fail(c, e, "phprng_skip: table allocation");
    }
    std::string err;
    int rc = launch_build_skip_table(c->p, c->a, c->d_T, c->d_P, seg, s, &err);
    cudaError_t e2 = cudaStreamSynchronize(s);                 // host copies, seg lifetime
    cudaFree(seg);
    if (rc != PHPRNG_OK) return fail(c, rc, "phprng_skip: " + err);
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "phprng_skip: table build");
    tb.T = c->d_T;
    tb.P = c->d_P;
    c->tbl = tb;
    c->skip_ready = true;
    return PHPRNG_OK;
}

// Pref(t) = sum_{i=1..t} (a^i mod p), 0 <= t <= p-1, on the host from the
// device table's checkpoint at floor(t/B) B plus the tail of fewer than B terms.
static int host_pref(phprng_ctx *c, uint64_t t, uint64_t *out)
{
    const uint64_t j = t >> kSkipLog2B;
    uint64_t T;
    uint32_t x;
    cudaError_t e = cudaMemcpy(&T, c->d_T + j, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&x, c->d_P + j, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "phprng_set_state: prefix table read");
    uint64_t v = x;
    for (uint64_t u = j << kSkipLog2B; u < t; ++u) {
        v = v * c->a % c->p;
        T += v;
    }
    *out = T;
    return PHPRNG_OK;
}

PH_API int phprng_set_state(phprng_ctx *ctx, uint64_t inst, uint64_t m, uint64_t s, uint64_t c,
                            uint64_t pos, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_set_state: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_set_state: a server owns the context");
    if (inst >= ctx->count) return fail(ctx, PHPRNG_EINVAL, "phprng_set_state: instance out of range");
    const uint64_t n = ctx->host_inst[inst].n, p = ctx->p, pm1 = p - 1;
    if (m >= n || c >= n) return fail(ctx, PHPRNG_EINVAL, "phprng_set_state: need m < n and c < n");
    if (s < 1 || s > pm1) return fail(ctx, PHPRNG_EINVAL, "phprng_set_state: need 1 <= s <= p-1");
    CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint64_t v[4] = {m, s, c, pos};
    if (ctx->wide_skip) {
        // a wide skip prime moves streams by stepping from the current state,
        // so the state alone defines the stream from here on
        CU(ctx, cudaStreamSynchronize(st));
        for (int k = 0; k < 4; ++k)
            CU(ctx, cudaMemcpy(ctx->d_state + (uint64_t)k * ctx->count + inst, &v[k], 8, cudaMemcpyHostToDevice));
        ctx->pos_host[inst] = pos;
        return PHPRNG_OK;
    }
    int rc = ensure_skip(ctx, st);
    if (rc != PHPRNG_OK) return rc;
    if (ctx->tbl.kind == 1) {
        // constant skip through (m, s = b) at pos: seed m0 = m - pos b mod n, s0 = b
        const uint64_t F = mulmod(pos % n, s % n, n);
        const uint64_t m0 = m >= F ? m - F : m + (n - F);
        CU(ctx, cudaStreamSynchronize(st));
        for (int k = 0; k < 4; ++k)
            CU(ctx, cudaMemcpy(ctx->d_state + (uint64_t)k * ctx->count + inst, &v[k], 8, cudaMemcpyHostToDevice));
        CU(ctx, cudaMemcpy(ctx->d_L0 + inst, &s, 8, cudaMemcpyHostToDevice));
        CU(ctx, cudaMemcpy(ctx->d_m0 + inst, &m0, 8, cudaMemcpyHostToDevice));
        ctx->host_inst[inst].m0 = m0;
        ctx->host_inst[inst].s0 = s;
        ctx->pos_host[inst] = pos;
        return PHPRNG_OK;
    }
    // the stream through (m, s) at position pos: cycle position of s, then the
    // seed pos steps earlier (Eq. 7 backwards: L0 = L - pos, m0 = m - F)
    uint64_t Ls;
    if (!discrete_logs(p, ctx->a, &s, 1, &Ls))
        return fail(ctx, PHPRNG_ESKIP, "phprng_set_state: no discrete log for s");
    const uint64_t q = pos / pm1, r = pos % pm1;
    const uint64_t L0 = (Ls + pm1 - r) % pm1;
    uint64_t P0, P1, W;
    rc = host_pref(ctx, L0, &P0);
    if (rc == PHPRNG_OK) rc = host_pref(ctx, L0 + r <= pm1 ? L0 + r : L0 + r - pm1, &P1);
    if (rc != PHPRNG_OK) return rc;
    W = L0 + r <= pm1 ? P1 - P0 : ctx->tbl.half - P0 + P1;
    const uint64_t F = (mulmod(q % n, ctx->tbl.half % n, n) + W % n) % n;
    const uint64_t m0 = m >= F ? m - F : m + (n - F), s0 = powmod(ctx->a, L0, p);
    CU(ctx, cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k)
        CU(ctx, cudaMemcpy(ctx->d_state + (uint64_t)k * ctx->count + inst, &v[k], 8, cudaMemcpyHostToDevice));
    CU(ctx, cudaMemcpy(ctx->d_L0 + inst, &L0, 8, cudaMemcpyHostToDevice));
    CU(ctx, cudaMemcpy(ctx->d_m0 + inst, &m0, 8, cudaMemcpyHostToDevice));
    ctx->host_inst[inst].m0 = m0;
    ctx->host_inst[inst].s0 = s0;
    ctx->pos_host[inst] = pos;
    return PHPRNG_OK;
}

// Skip requests of a context with a wide skip prime, one after another: the
// window sums are formed by stepping, so r = k mod (p-1) is bounded per call.
static constexpr uint64_t kWideSkipMaxSteps = 1ull << 40;

static int run_wide_skips(phprng_ctx *ctx, const std::vector<SkipReq> &reqs, cudaStream_t s,
                          const char *what)
{
    const std::string w(what);
    for (const SkipReq &r : reqs)
        if (r.k % (ctx->p - 1) > kWideSkipMaxSteps)
            return fail(ctx, PHPRNG_EINVAL, w + ": with a skip prime p >= 2^32 the steps beyond whole "
                                                "cycles of p-1 are formed one by one; at most 2^40 per call");
    uint64_t *scratch = nullptr;
    CU(ctx, cudaMallocAsync((void **)&scratch, (1 + phprng::kWideSkipBlocks) * sizeof(uint64_t), s));
    std::string err;
    int rc = PHPRNG_OK;
    for (const SkipReq &r : reqs) {
        rc = launch_skip_wide(ctx->d_inst, ctx->d_prog, ctx->st, ctx->skw64, ctx->ainvM, r, scratch, s, &err);
        if (rc != PHPRNG_OK) break;
    }
    cudaError_t e = cudaFreeAsync(scratch, s);
    if (rc != PHPRNG_OK) return fail(ctx, rc, w + ": " + err);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFreeAsync");
    return PHPRNG_OK;
}

PH_API int phprng_skip(phprng_ctx *ctx, const uint64_t *inst_ids, const uint64_t *k,
                       uint64_t cnt, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_skip: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_skip: a server owns the context");
    if (cnt == 0) return PHPRNG_OK;
    if (!inst_ids || !k) return fail(ctx, PHPRNG_EINVAL, "phprng_skip: NULL request arrays");
    // merge repeated instances (their skips add) and check for overflow
    std::vector<SkipReq> reqs;
    std::vector<uint64_t> slot;
    try {
        reqs.reserve(cnt);
        slot.assign(ctx->count, UINT64_MAX);
    } catch (const std::bad_alloc &) {
        return fail(ctx, PHPRNG_ENOMEM, "phprng_skip: host allocation failed");
    }
    for (uint64_t j = 0; j < cnt; ++j) {
        const uint64_t i = inst_ids[j];
        if (i >= ctx->count) return fail(ctx, PHPRNG_EINVAL, "phprng_skip: instance out of range");
        if (slot[i] == UINT64_MAX) {
            slot[i] = reqs.size();
            reqs.push_back({i, 0, 0});
        }
        SkipReq &r = reqs[slot[i]];
        if (k[j] > UINT64_MAX - r.k || r.k + k[j] > UINT64_MAX - ctx->pos_host[i])
            return fail(ctx, PHPRNG_EINVAL, "phprng_skip: stream position would exceed 2^64-1");
        r.k += k[j];
    }
    CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (ctx->wide_skip) {
        int wrc = run_wide_skips(ctx, reqs, s, "phprng_skip");
        if (wrc != PHPRNG_OK) return wrc;
        for (const SkipReq &r : reqs) ctx->pos_host[r.inst] += r.k;
        return PHPRNG_OK;
    }
    int rc = ensure_skip(ctx, s);
    if (rc != PHPRNG_OK) return rc;
    SkipReq *d_reqs = nullptr;
    CU(ctx, cudaMallocAsync((void **)&d_reqs, reqs.size() * sizeof(SkipReq), s));
    cudaError_t e = cudaMemcpyAsync(d_reqs, reqs.data(), reqs.size() * sizeof(SkipReq),
                                    cudaMemcpyHostToDevice, s);
    std::string err;
    if (e == cudaSuccess)
        rc = launch_skip(ctx->d_inst, ctx->d_prog, ctx->st, ctx->d_L0, ctx->tbl, d_reqs, reqs.size(), s, &err);
    cudaError_t e2 = cudaFreeAsync(d_reqs, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "phprng_skip: request upload");
    if (rc != PHPRNG_OK) return fail(ctx, rc, "phprng_skip: " + err);
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "phprng_skip: cudaFreeAsync");
    // the pageable upload above completes before cudaMemcpyAsync returns
    for (const SkipReq &r : reqs) ctx->pos_host[r.inst] += r.k;
    return PHPRNG_OK;
}

// Shared by the serial, poker and runs tests: validation of the range, the
// launch, the positions.  D = 0 selects the poker test, D = -1 the runs test
// (B = lmax).
static int run_hist_test(phprng_ctx *ctx, const char *what, uint64_t first, uint64_t num_inst,
                         uint64_t per_inst, int D, uint32_t B, uint64_t *hist, void *cuda_stream,
                         const std::function<int(const GenArgs &, cudaStream_t, std::string *)> &launch =
                             nullptr)
{
    const std::string w(what);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, w + ": a server owns the context");
    if (first > ctx->count || num_inst > ctx->count - first)
        return fail(ctx, PHPRNG_EINVAL, w + ": instance range outside the table");
    if (!hist || (uintptr_t)hist % 8)
        return fail(ctx, PHPRNG_EINVAL, w + ": hist NULL or not 8-byte aligned");
    if (num_inst == 0 || per_inst == 0) return PHPRNG_OK;
    for (uint64_t i = first; i < first + num_inst; ++i)
        if (ctx->wide[i]) return fail(ctx, PHPRNG_EINVAL, w + ": defined for 32-bit moduli only");
    CU(ctx, cudaSetDevice(ctx->device));
    if (pointer_kind(hist) != 1) return fail(ctx, PHPRNG_EINVAL, w + ": hist must be device memory");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    GenArgs g;
    g.inst = ctx->d_inst;
    g.prog = ctx->d_prog;
    g.prog8 = ctx->d_prog8;
    g.st = ctx->st;
    g.sk = ctx->sk32_8;
    g.first = first;
    g.num = num_inst;
    g.per_inst = per_inst;
    g.c_out = nullptr;
    g.r_out = nullptr;
    g.stats = nullptr;
    g.edge = nullptr;
    g.c_is_64 = 0;
    g.vec_ok = 0;
    if (num_inst >= kOrderMinInstances && num_inst < (1ull << 32)) {
        int rc = PHPRNG_OK;
        g.order = instance_order(ctx, first, num_inst, s, &rc);
        if (rc != PHPRNG_OK) return rc;
    }
    std::string err;
    int rc = launch ? launch(g, s, &err)
             : D < 0 ? launch_runs(g, (int)B, (unsigned long long *)hist, s, &err)
                     : launch_serial(g, D, B, (unsigned long long *)hist, s, &err);
    if (rc != PHPRNG_OK) return fail(ctx, rc, w + ": " + err);
    for (uint64_t i = first; i < first + num_inst; ++i) ctx->pos_host[i] += per_inst;
    return PHPRNG_OK;
}

PH_API int phprng_serial_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                              int D, uint32_t B, uint64_t *hist, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_serial_test: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (D < 1 || D > 8) return fail(ctx, PHPRNG_EINVAL, "phprng_serial_test: D must be 1..8");
    const bool pow2 = B && (B & (B - 1)) == 0;
    if (B < 1 || (pow2 ? B > (1u << 20) : B > (1u << 16)))
        return fail(ctx, PHPRNG_EINVAL,
                    "phprng_serial_test: B must be a power of two up to 2^20 or at most 2^16");
    uint64_t bins = 1;
    for (int d = 0; d < D; ++d) bins *= B;
    if (bins > (1ull << 24)) return fail(ctx, PHPRNG_EINVAL, "phprng_serial_test: B^D exceeds 2^24");
    return run_hist_test(ctx, "phprng_serial_test", first, num_inst, per_inst, D, B, hist, cuda_stream);
}

PH_API int phprng_poker_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                             uint64_t *hist, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_poker_test: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    return run_hist_test(ctx, "phprng_poker_test", first, num_inst, per_inst, 0, 10, hist, cuda_stream);
}

PH_API int phprng_collision_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                                 uint32_t S, uint32_t B, uint32_t H, uint64_t *hist, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_collision_test: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (S < 256 || S % 256 || S > (1u << 24))
        return fail(ctx, PHPRNG_EINVAL,
                    "phprng_collision_test: S must be a multiple of 256 from 256 to 2^24");
    const bool pow2 = B && (B & (B - 1)) == 0;
    if (B < 1 || (pow2 ? B > (1u << 20) : B > (1u << 16)))
        return fail(ctx, PHPRNG_EINVAL,
                    "phprng_collision_test: B must be a power of two up to 2^20 or at most 2^16");
    if (H < 1 || H > (1u << 16)) return fail(ctx, PHPRNG_EINVAL, "phprng_collision_test: H must be 1..2^16");
    auto launch = [&](const GenArgs &g, cudaStream_t s, std::string *err) -> int {
        // scratch for the bins of at most kCollBinsCap numbers at a time
        const uint64_t counted = per_inst / S * S;
        const uint64_t want = counted > kCollBinsCap / num_inst ? kCollBinsCap : counted * num_inst;
        const uint64_t cap = std::max<uint64_t>(S, std::min<uint64_t>(kCollBinsCap, want));
        uint32_t *bins = nullptr;
        if (counted) {
            cudaError_t e = cudaMallocAsync((void **)&bins, cap * sizeof(uint32_t), s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                *err = std::string("collision bins: ") + cudaGetErrorString(e);
                return e == cudaErrorMemoryAllocation ? PHPRNG_ENOMEM : PHPRNG_ECUDA;
            }
        }
        int rc = launch_collision(g, S, B, H, (unsigned long long *)hist, bins, cap, s, err);
        if (bins) cudaFreeAsync(bins, s);
        return rc;
    };
    return run_hist_test(ctx, "phprng_collision_test", first, num_inst, per_inst, 1, 1, hist, cuda_stream,
                         launch);
}

PH_API int phprng_interstream_serial_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst,
                                         uint64_t per_inst, int D, uint32_t B, uint64_t *hist,
                                         void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_interstream_serial_test: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    const char *W = "phprng_interstream_serial_test: ";
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, std::string(W) + "a server owns the context");
    if (first > ctx->count || num_inst > ctx->count - first)
        return fail(ctx, PHPRNG_EINVAL, std::string(W) + "instance range outside the table");
    if (D < 1 || D > 8) return fail(ctx, PHPRNG_EINVAL, std::string(W) + "D must be 1..8");
    const bool pow2 = B && (B & (B - 1)) == 0;
    if (B < 1 || (pow2 ? B > (1u << 20) : B > (1u << 16)))
        return fail(ctx, PHPRNG_EINVAL, std::string(W) + "B must be a power of two up to 2^20 or at most 2^16");
    uint64_t bins = 1;
    for (int d = 0; d < D; ++d) bins *= B;
    if (bins > (1ull << 24)) return fail(ctx, PHPRNG_EINVAL, std::string(W) + "B^D exceeds 2^24");
    if (!hist || (uintptr_t)hist % 8) return fail(ctx, PHPRNG_EINVAL, std::string(W) + "hist NULL or misaligned");
    if (num_inst == 0 || per_inst == 0) return PHPRNG_OK;
    for (uint64_t i = first; i < first + num_inst; ++i)
        if (ctx->wide[i]) return fail(ctx, PHPRNG_EINVAL, std::string(W) + "defined for 32-bit moduli only");
    CU(ctx, cudaSetDevice(ctx->device));
    if (pointer_kind(hist) != 1) return fail(ctx, PHPRNG_EINVAL, std::string(W) + "hist must be device memory");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool groups = D >= 2;                          // 2 <= D <= 8
    if (ctx->width == 32 && D == 1) {
        // single numbers: the interleaved order does not change their
        // histogram, which is the frequency test's (serial kernel, D = 1)
        GenArgs g;
        g.inst = ctx->d_inst;
        g.prog = ctx->d_prog;
        g.prog8 = ctx->d_prog8;
        g.st = ctx->st;
        g.sk = ctx->sk32_8;
        g.first = first;
        g.num = num_inst;
        g.per_inst = per_inst;
        int rc = PHPRNG_OK;
        if (num_inst >= kOrderMinInstances && num_inst < (1ull << 32))
            g.order = instance_order(ctx, first, num_inst, s, &rc);
        if (rc != PHPRNG_OK) return rc;
        std::string err;
        rc = launch_serial(g, 1, B, (unsigned long long *)hist, s, &err);
        if (rc != PHPRNG_OK) return fail(ctx, rc, std::string(W) + err);
        for (uint64_t i = first; i < first + num_inst; ++i) ctx->pos_host[i] += per_inst;
        return PHPRNG_OK;
    }
    if (ctx->width == 32 && B <= (1u << 16) && groups && num_inst % (uint64_t)D == 0) {
        // Groups of D streams as adjacent warps, their tuples counted as they
        // are generated; group slots heaviest first (the heaviest of the D
        // exponent programs)
        const uint64_t ng = num_inst / (uint64_t)D;
        uint32_t *gord = nullptr;
        if (ng >= kOrderMinInstances / (uint64_t)D && ng < (1ull << 32)) {
            std::vector<uint32_t> ord(ng), cnt(513, 0);
            auto gkey = [&](uint64_t q) {
                uint16_t k = ctx->key[first + (uint64_t)D * q];
                for (int d = 1; d < D; ++d) k = std::min(k, ctx->key[first + (uint64_t)D * q + d]);
                return k;
            };
            for (uint64_t q = 0; q < ng; ++q) ++cnt[gkey(q) + 1];
            for (int k = 1; k <= 512; ++k) cnt[k] += cnt[k - 1];
            for (uint64_t q = 0; q < ng; ++q) ord[cnt[gkey(q)]++] = (uint32_t)q;
            cudaError_t e = cudaMallocAsync((void **)&gord, ng * sizeof(uint32_t), s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(gord, ord.data(), ng * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (gord) cudaFreeAsync(gord, s);
                return fail(ctx, PHPRNG_ENOMEM, std::string(W) + "group order upload failed");
            }
        }
        GenArgs g;
        g.inst = ctx->d_inst;
        g.prog = ctx->d_prog;
        g.prog8 = ctx->d_prog8;
        g.st = ctx->st;
        g.sk = ctx->sk32_8;
        g.first = first;
        g.num = num_inst;
        g.per_inst = per_inst;
        std::string err;
        const int rc = launch_inter_groups(g, D, B, (unsigned long long *)hist, gord, s, &err);
        if (gord) cudaFreeAsync(gord, s);
        if (rc != PHPRNG_OK) return fail(ctx, rc, std::string(W) + err);
        for (uint64_t i = first; i < first + num_inst; ++i) ctx->pos_host[i] += per_inst;
        return PHPRNG_OK;
    }
    // chunks of Lch numbers per stream, a multiple of D so that no tuple of the
    // interleaved sequence spans two chunks; about 2^25 numbers per chunk
    uint64_t Lch = (1ull << 25) / num_inst / (uint64_t)D * (uint64_t)D;
    if (Lch < (uint64_t)D) Lch = (uint64_t)D;
    if (Lch > kInterMaxChunk) Lch = kInterMaxChunk / (uint64_t)D * (uint64_t)D;
    if (Lch > per_inst) Lch = per_inst;
    const int c64 = ctx->width != 32;                   // c's element size as launch_range writes it
    void *c = nullptr, *kc = nullptr;
    uint32_t *binsT = nullptr;
    cudaError_t e = cudaMallocAsync(&c, num_inst * Lch * (c64 ? 8 : 4), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&binsT, num_inst * Lch * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&kc, num_inst * 16, s);
    std::string err;
    int rc = e == cudaSuccess ? PHPRNG_OK : PHPRNG_ENOMEM;
    if (rc == PHPRNG_OK) rc = launch_inter_consts(ctx->d_inst, first, num_inst, B, kc, s, &err);
    for (uint64_t j0 = 0; j0 < per_inst && rc == PHPRNG_OK; j0 += Lch) {
        const uint64_t L = std::min(Lch, per_inst - j0);
        rc = launch_range(ctx, first, num_inst, L, c, nullptr, nullptr, s, true);   // Eq. 9
        if (rc != PHPRNG_OK) break;
        rc = launch_interstream(kc, num_inst, L, c, c64, D, B, binsT,
                                (unsigned long long *)hist, s, &err);
        if (rc == PHPRNG_OK)
            for (uint64_t i = first; i < first + num_inst; ++i) ctx->pos_host[i] += L;
    }
    if (c) cudaFreeAsync(c, s);
    if (binsT) cudaFreeAsync(binsT, s);
    if (kc) cudaFreeAsync(kc, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PHPRNG_ENOMEM, std::string(W) + "scratch allocation failed");
    }
    if (rc != PHPRNG_OK) return err.empty() ? rc : fail(ctx, rc, std::string(W) + err);
    return PHPRNG_OK;
}

PH_API int phprng_fourier_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                               uint32_t log2M, uint32_t nbins, double w, uint64_t *hist, double *coef_out,
                               void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_fourier_test: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: a server owns the context");
    if (first > ctx->count || num_inst > ctx->count - first)
        return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: instance range outside the table");
    if (log2M < 2 || log2M > 20) return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: log2M must be 2..20");
    const uint64_t M = 1ull << log2M;
    if (per_inst % M) return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: per_inst must be a multiple of M");
    if (nbins < 1 || nbins > (1u << 24) || !(w > 0.0) || !(w < 1e300))
        return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: need 1 <= nbins <= 2^24 and w > 0");
    if (!hist || (uintptr_t)hist % 8 || (uintptr_t)coef_out % 16)
        return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: hist NULL or misaligned, or coef_out misaligned");
    if (num_inst == 0 || per_inst == 0) return PHPRNG_OK;
    for (uint64_t i = first; i < first + num_inst; ++i)
        if (ctx->wide[i]) return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: defined for 32-bit moduli only");
    CU(ctx, cudaSetDevice(ctx->device));
    if (pointer_kind(hist) != 1 || (coef_out && pointer_kind(coef_out) != 1))
        return fail(ctx, PHPRNG_EINVAL, "phprng_fourier_test: hist and coef_out must be device memory");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // instances per batch: R scratch of at most 2^26 doubles (512 MiB)
    const uint64_t batch = std::max<uint64_t>(1, std::min<uint64_t>(num_inst, (1ull << 26) / per_inst));
    double2 *tw = nullptr, *Z = nullptr;
    double *R = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&tw, fourier_twiddle_count(log2M) * sizeof(double2), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&R, batch * per_inst * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&Z, batch * per_inst / 2 * sizeof(double2), s);
    std::string err;
    int rc = e == cudaSuccess ? PHPRNG_OK : PHPRNG_ENOMEM;
    const double scale2 = 0.5 / std::sqrt((double)M);
    if (rc == PHPRNG_OK) rc = launch_twiddles(tw, log2M, scale2, s, &err);
    for (uint64_t b0 = 0; b0 < num_inst && rc == PHPRNG_OK; b0 += batch) {
        const uint64_t nb = std::min(batch, num_inst - b0);
        rc = launch_range(ctx, first + b0, nb, per_inst, nullptr, R, nullptr, s, true);   // Eq. 9
        if (rc != PHPRNG_OK) break;
        double *cb = coef_out ? coef_out + 2 * (b0 * per_inst / 2) : nullptr;
        rc = launch_fourier(R, nb * per_inst / M, log2M, tw, Z, nbins, w, scale2, hist, cb, s, &err);
        if (rc == PHPRNG_OK)
            for (uint64_t i = first + b0; i < first + b0 + nb; ++i) ctx->pos_host[i] += per_inst;
    }
    if (tw) cudaFreeAsync(tw, s);
    if (R) cudaFreeAsync(R, s);
    if (Z) cudaFreeAsync(Z, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PHPRNG_ENOMEM, "phprng_fourier_test: scratch allocation failed");
    }
    if (rc != PHPRNG_OK) return err.empty() ? rc : fail(ctx, rc, "phprng_fourier_test: " + err);
    return PHPRNG_OK;
}

PH_API int phprng_runs_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                            int lmax, uint64_t *hist, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_runs_test: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (lmax < 1 || lmax > 64) return fail(ctx, PHPRNG_EINVAL, "phprng_runs_test: lmax must be 1..64");
    if (per_inst >= (1ull << 32))
        return fail(ctx, PHPRNG_EINVAL, "phprng_runs_test: per_inst must be below 2^32");
    return run_hist_test(ctx, "phprng_runs_test", first, num_inst, per_inst, -1, (uint32_t)lmax, hist,
                         cuda_stream);
}

// e^-1 mod m (gcd(e, m) = 1) by the extended Euclidean algorithm.
static uint64_t inverse_mod(uint64_t e, uint64_t m)
{
    __int128 r0 = m, r1 = e % m, t0 = 0, t1 = 1;
    while (r1) {
        const __int128 q = r0 / r1;
        __int128 tmp = r0 - q * r1;
        r0 = r1;
        r1 = tmp;
        tmp = t0 - q * t1;
        t0 = t1;
        t1 = tmp;
    }
    return (uint64_t)(t0 < 0 ? t0 + m : t0);
}

static int pattern_impl(const char *name, const phprng_instance *inst, uint64_t c_lo, uint64_t L0, int D,
                        uint32_t nb, uint32_t L1, uint64_t *hist, void *cuda_stream)
{
    const std::string W = std::string(name) + ": ";
    if (!inst) return fail(nullptr, PHPRNG_EINVAL, W + "inst is NULL");
    phprng_instance in = *inst;
    in.m0 = 0;                                               // the seeds play no part
    in.s0 = 1;
    std::string msg;
    int rc = validate_one(32, in, 0, &msg);
    if (rc != PHPRNG_OK) return fail(nullptr, rc, W + msg);
    inst = &in;
    const uint64_t n = inst->n;
    if (L0 < 1 || L0 > (1ull << 20) || c_lo >= n || L0 > n - c_lo)
        return fail(nullptr, PHPRNG_EINVAL,
                    W + "need 1 <= L0 <= 2^20 and c_lo + L0 <= n");
    if (D < 2 || D > 8) return fail(nullptr, PHPRNG_EINVAL, W + "D must be 2..8");
    uint64_t bins = 1;
    for (int d = 1; d < D && bins <= (1ull << 24); ++d) bins *= nb;
    if (nb < 1 || bins > (1ull << 24))
        return fail(nullptr, PHPRNG_EINVAL, W + "nb^(D-1) must be 1 .. 2^24");
    if (!hist || (uintptr_t)hist % 8)
        return fail(nullptr, PHPRNG_EINVAL, W + "hist NULL or not 8-byte aligned");
    if (pointer_kind(hist) != 1)
        return fail(nullptr, PHPRNG_EINVAL, W + "hist must be device memory");
    ExpProg pg;
    const DevInst P = derive_inst(*inst, 0, &pg);
    const SkipConst sk = derive_skip(inst->p, inst->a, 8);
    const uint64_t d = inverse_mod(inst->e, n - 1);            // Eq. 2
    std::vector<uint32_t> mtab;
    try {
        mtab.resize(L0);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, PHPRNG_ENOMEM, W + "host allocation failed");
    }
    for (uint64_t q = 0; q < L0; ++q) mtab[q] = (uint32_t)powmod(c_lo + q, d, n);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t *d_m = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d_m, L0 * sizeof(uint32_t), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, PHPRNG_ENOMEM, W + "device allocation failed");
    }
    // from pageable memory: staged before the call returns, then ordered on s
    e = cudaMemcpyAsync(d_m, mtab.data(), L0 * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    std::string err;
    rc = e == cudaSuccess ? launch_pattern(P, pg, sk, d_m, L0, D, nb, L1, hist, s, &err) : PHPRNG_ECUDA;
    cudaFreeAsync(d_m, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, (W + "upload").c_str());
    if (rc != PHPRNG_OK) return fail(nullptr, rc, W + err);
    return PHPRNG_OK;
}

PH_API int phprng_pattern(const phprng_instance *inst, uint64_t c_lo, uint64_t L0, int D, uint32_t nb,
                          uint64_t *hist, void *cuda_stream)
{
    return pattern_impl("phprng_pattern", inst, c_lo, L0, D, nb, 0, hist, cuda_stream);
}

PH_API int phprng_pattern_region(const phprng_instance *inst, uint64_t c_lo, uint64_t L0, int D, uint32_t nb,
                                 uint32_t L1, uint64_t *hist, void *cuda_stream)
{
    if (L1 < 1) return fail(nullptr, PHPRNG_EINVAL, "phprng_pattern_region: L1 must be at least 1");
    return pattern_impl("phprng_pattern_region", inst, c_lo, L0, D, nb, L1, hist, cuda_stream);
}

static int pattern_const_impl(const char *name, const phprng_instance *inst, uint64_t b, uint64_t c_lo,
                              uint64_t L0, int D, uint32_t nb, uint32_t L1, uint64_t *hist, void *cuda_stream)
{
    const std::string W = std::string(name) + ": ";
    if (!inst) return fail(nullptr, PHPRNG_EINVAL, W + "inst is NULL");
    phprng_instance in = *inst;
    in.p = 3;                                                // only n and e play a part:
    in.a = 2;                                                // a valid stand-in skip generator
    in.m0 = 0;
    in.s0 = 1;
    std::string msg;
    int rc = validate_one(32, in, 0, &msg);
    if (rc != PHPRNG_OK) return fail(nullptr, rc, W + msg);
    const uint64_t n = in.n;
    if (b < 1 || b >= n) return fail(nullptr, PHPRNG_EINVAL, W + "need 1 <= b < n");
    if (L0 < 1 || c_lo >= n || L0 > n - c_lo)
        return fail(nullptr, PHPRNG_EINVAL, W + "need L0 >= 1 and c_lo + L0 <= n");
    if (D < 2 || D > 8) return fail(nullptr, PHPRNG_EINVAL, W + "D must be 2..8");
    uint64_t bins = 1;
    for (int d = 1; d < D && bins <= (1ull << 24); ++d) bins *= nb;
    if (nb < 1 || bins > (1ull << 24))
        return fail(nullptr, PHPRNG_EINVAL, W + "nb^(D-1) must be 1 .. 2^24");
    if (!hist || (uintptr_t)hist % 8)
        return fail(nullptr, PHPRNG_EINVAL, W + "hist NULL or not 8-byte aligned");
    if (pointer_kind(hist) != 1)
        return fail(nullptr, PHPRNG_EINVAL, W + "hist must be device memory");
    ExpProg pg, pgd;
    const DevInst P = derive_inst(in, 0, &pg);
    phprng_instance dec = in;
    dec.e = inverse_mod(in.e, n - 1);                        // Eq. 2
    const DevInst Pd = derive_inst(dec, 0, &pgd);
    std::string err;
    rc = launch_pattern_const(P, pg, Pd, pgd, (uint32_t)b, c_lo, L0, D, nb, L1, hist, cuda_stream, &err);
    if (rc != PHPRNG_OK) return fail(nullptr, rc, W + err);
    return PHPRNG_OK;
}

PH_API int phprng_pattern_const(const phprng_instance *inst, uint64_t b, uint64_t c_lo, uint64_t L0,
                                int D, uint32_t nb, uint64_t *hist, void *cuda_stream)
{
    return pattern_const_impl("phprng_pattern_const", inst, b, c_lo, L0, D, nb, 0, hist, cuda_stream);
}

PH_API int phprng_pattern_const_region(const phprng_instance *inst, uint64_t b, uint64_t c_lo, uint64_t L0,
                                       int D, uint32_t nb, uint32_t L1, uint64_t *hist, void *cuda_stream)
{
    if (L1 < 1) return fail(nullptr, PHPRNG_EINVAL, "phprng_pattern_const_region: L1 must be at least 1");
    return pattern_const_impl("phprng_pattern_const_region", inst, b, c_lo, L0, D, nb, L1, hist, cuda_stream);
}

PH_API int phprng_seek(phprng_ctx *ctx, const uint64_t *inst_ids, const uint64_t *pos,
                       uint64_t cnt, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_seek: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_seek: a server owns the context");
    if (cnt == 0) return PHPRNG_OK;
    if (!inst_ids || !pos) return fail(ctx, PHPRNG_EINVAL, "phprng_seek: NULL request arrays");
    std::vector<SkipReq> reqs;
    std::vector<uint64_t> slot;
    try {
        reqs.reserve(cnt);
        slot.assign(ctx->count, UINT64_MAX);
    } catch (const std::bad_alloc &) {
        return fail(ctx, PHPRNG_ENOMEM, "phprng_seek: host allocation failed");
    }
    std::vector<uint64_t> target;
    for (uint64_t j = 0; j < cnt; ++j) {                // the last target of an instance wins
        const uint64_t i = inst_ids[j];
        if (i >= ctx->count) return fail(ctx, PHPRNG_EINVAL, "phprng_seek: instance out of range");
        if (slot[i] == UINT64_MAX) {
            slot[i] = reqs.size();
            reqs.push_back({i, 0, 0});
            target.push_back(0);
        }
        target[slot[i]] = pos[j];
    }
    for (size_t r = 0; r < reqs.size(); ++r) {
        const uint64_t cur = ctx->pos_host[reqs[r].inst];
        reqs[r].back = target[r] < cur ? 1 : 0;
        reqs[r].k = target[r] < cur ? cur - target[r] : target[r] - cur;
    }
    CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (ctx->wide_skip) {
        int wrc = run_wide_skips(ctx, reqs, s, "phprng_seek");
        if (wrc != PHPRNG_OK) return wrc;
        for (size_t r = 0; r < reqs.size(); ++r) ctx->pos_host[reqs[r].inst] = target[r];
        return PHPRNG_OK;
    }
    int rc = ensure_skip(ctx, s);
    if (rc != PHPRNG_OK) return rc;
    SkipReq *d_reqs = nullptr;
    CU(ctx, cudaMallocAsync((void **)&d_reqs, reqs.size() * sizeof(SkipReq), s));
    cudaError_t e = cudaMemcpyAsync(d_reqs, reqs.data(), reqs.size() * sizeof(SkipReq),
                                    cudaMemcpyHostToDevice, s);
    std::string err;
    if (e == cudaSuccess)
        rc = launch_skip(ctx->d_inst, ctx->d_prog, ctx->st, ctx->d_L0, ctx->tbl, d_reqs, reqs.size(), s, &err);
    cudaError_t e2 = cudaFreeAsync(d_reqs, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "phprng_seek: request upload");
    if (rc != PHPRNG_OK) return fail(ctx, rc, "phprng_seek: " + err);
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "phprng_seek: cudaFreeAsync");
    for (size_t r = 0; r < reqs.size(); ++r) ctx->pos_host[reqs[r].inst] = target[r];
    return PHPRNG_OK;
}

PH_API int phprng_microbench(int which, double *ops_per_s, void *cuda_stream)
{
    if (!ops_per_s) return fail(nullptr, PHPRNG_EINVAL, "phprng_microbench: ops_per_s is NULL");
    std::string err;
    int rc = run_microbench(which, ops_per_s, cuda_stream, &err);
    if (rc != PHPRNG_OK) return fail(nullptr, rc, err);
    return PHPRNG_OK;
}

// ---- batches ----------------------------------------------------------------

struct phprng_plan {
    struct Req {
        uint64_t inst, start, len, c_off, r_off;
        bool last;                         // last request of its instance
    };
    phprng_ctx *ctx = nullptr;
    std::vector<Req> reqs;
    std::vector<std::pair<uint64_t, uint64_t>> final_pos;   // (instance, position after)
    Tile *d_tiles = nullptr;
    size_t tiles_cap = 0;
    uint64_t ntiles = 0;
    unsigned long long *d_counter = nullptr;
    phprng_tuning tune{};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    void *g_c = nullptr;
    double *g_r = nullptr;
};

static const uint32_t kDefaultTile = 16384;

static void free_plan(phprng_plan *pl)
{
    if (!pl) return;
    cudaDeviceSynchronize();
    if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    cudaFree(pl->d_tiles);
    cudaFree(pl->d_counter);
    delete pl;
}

// Cuts the resolved requests into tiles, heaviest first, and uploads them.
static int build_tiles(phprng_plan *pl, uint32_t tile)
{
    phprng_ctx *c = pl->ctx;
    std::vector<Tile> t;
    for (const auto &r : pl->reqs) {
        const uint32_t wide = c->wide[r.inst] ? kTileWide : 0u;
        for (uint64_t k = 0; k < r.len; k += tile) {
            Tile x;
            x.len = (uint32_t)std::min<uint64_t>(tile, r.len - k);
            x.inst = (uint32_t)r.inst | wide | ((r.last && k + x.len == r.len) ? kTileWriteBack : 0u);
            x.start = r.start + k;
            x.c_off = r.c_off + k;
            x.r_off = r.r_off + k;
            t.push_back(x);
        }
    }
    std::stable_sort(t.begin(), t.end(), [](const Tile &a, const Tile &b) {
        const bool wa = (a.inst & kTileWide) != 0, wb = (b.inst & kTileWide) != 0;
        if (wa != wb) return wa;
        return a.len > b.len;
    });
    if (t.size() > pl->tiles_cap) {
        cudaFree(pl->d_tiles);
        pl->d_tiles = nullptr;
        pl->tiles_cap = 0;
        cudaError_t e = cudaMalloc(&pl->d_tiles, t.size() * sizeof(Tile));
        if (e != cudaSuccess) return cuda_fail(c, e, "phprng_plan: tile list allocation");
        pl->tiles_cap = t.size();
    }
    if (!t.empty())
        CU(c, cudaMemcpy(pl->d_tiles, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    pl->ntiles = t.size();
    pl->tune.tile = tile;
    if (pl->gexec) {                                  // the captured graph names the old list
        cudaGraphExecDestroy(pl->gexec);
        pl->gexec = nullptr;
    }
    return PHPRNG_OK;
}

static BatchArgs batch_args(phprng_plan *pl, void *c_base, double *r_base)
{
    phprng_ctx *c = pl->ctx;
    BatchArgs a;
    a.inst = c->d_inst;
    a.prog = c->d_prog;
    a.prog8 = c->d_prog8;
    a.st = c->st;
    a.m0 = c->d_m0;
    a.L0 = c->d_L0;
    a.tb = c->tbl;
    a.sk32_8 = c->sk32_8;
    a.sk32_4 = c->sk32_4;
    a.sk64 = c->sk64;
    a.tiles = pl->d_tiles;
    a.ntiles = pl->ntiles;
    a.counter = pl->d_counter;
    a.c_base = c_base;
    a.r_base = r_base;
    a.c_is_64 = c->width != 32;
    a.vec_ok = ((uintptr_t)c_base % 16 == 0) && ((uintptr_t)r_base % 16 == 0);
    return a;
}

PH_API int phprng_plan_create(phprng_ctx *ctx, const phprng_request *reqs, uint64_t nreq,
                              uint32_t tile, phprng_plan **out, void *cuda_stream)
{
    if (!out) return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: out is NULL");
    *out = nullptr;
    if (!ctx) return fail(nullptr, PHPRNG_EINVAL, "phprng_plan_create: ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: a server owns the context");
    if (ctx->wide_skip)
        return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: batched tiles start by Eq. 7 from the prefix "
                                        "table, which a skip prime p >= 2^32 does not have");
    if (nreq && !reqs) return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: reqs is NULL");
    if (tile == 0) tile = kDefaultTile;
    if (tile > (1u << 30)) return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: tile above 2^30");
    if (ctx->count > kTileInstMask)
        return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: more than 2^30 instances");
    phprng_plan *pl = new (std::nothrow) phprng_plan;
    if (!pl) return fail(ctx, PHPRNG_ENOMEM, "phprng_plan_create: host allocation failed");
    pl->ctx = ctx;
    pl->tune.npt = 8;
    pl->tune.blocks_per_sm = 0;
    try {
        std::vector<uint64_t> cursor(ctx->pos_host);
        std::vector<int64_t> lastreq(ctx->count, -1);
        pl->reqs.reserve(nreq);
        for (uint64_t j = 0; j < nreq; ++j) {
            const phprng_request &r = reqs[j];
            if (r.inst >= ctx->count) {
                delete pl;
                return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: request " + std::to_string(j) +
                                                    ": instance out of range");
            }
            if (r.len == 0) continue;                        // ignored entirely
            const uint64_t start = r.offset == PHPRNG_CONTINUE ? cursor[r.inst] : r.offset;
            if (r.len > UINT64_MAX - start || r.len > UINT64_MAX - r.c_off ||
                r.len > UINT64_MAX - r.r_off) {
                delete pl;
                return fail(ctx, PHPRNG_EINVAL, "phprng_plan_create: request " + std::to_string(j) +
                                                    ": position or offset overflow");
            }
            cursor[r.inst] = start + r.len;
            lastreq[r.inst] = (int64_t)pl->reqs.size();
            pl->reqs.push_back({r.inst, start, r.len, r.c_off, r.r_off, false});
        }
        for (uint64_t i = 0; i < ctx->count; ++i) {
            if (lastreq[i] >= 0) {
                pl->reqs[lastreq[i]].last = true;
                pl->final_pos.push_back({i, cursor[i]});
            }
        }
    } catch (const std::bad_alloc &) {
        delete pl;
        return fail(ctx, PHPRNG_ENOMEM, "phprng_plan_create: host allocation failed");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) { delete pl; return cuda_fail(ctx, e, "cudaSetDevice"); }
    int rc = ensure_skip(ctx, (cudaStream_t)cuda_stream);
    if (rc != PHPRNG_OK) { delete pl; return rc; }
    e = cudaMalloc(&pl->d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) { free_plan(pl); return cuda_fail(ctx, e, "phprng_plan_create: counter"); }
    rc = build_tiles(pl, tile);
    if (rc != PHPRNG_OK) { free_plan(pl); return rc; }
    *out = pl;
    return PHPRNG_OK;
}

static int plan_launch_locked(phprng_plan *pl, void *c_base, double *r_base, cudaStream_t s)
{
    phprng_ctx *c = pl->ctx;
    const size_t csz = c->width == 32 ? 4 : 8;
    if ((uintptr_t)c_base % csz || (uintptr_t)r_base % 8)
        return fail(c, PHPRNG_EINVAL, "phprng_plan_launch: output base not aligned to its element");
    std::string err;
    int rc = launch_batch(batch_args(pl, c_base, r_base), pl->tune.npt, pl->tune.blocks_per_sm, s, &err);
    if (rc != PHPRNG_OK) return fail(c, rc, "phprng_plan_launch: " + err);
    for (const auto &fp : pl->final_pos) c->pos_host[fp.first] = fp.second;
    return PHPRNG_OK;
}

PH_API int phprng_plan_launch(phprng_plan *plan, void *c_base, double *r_base, void *cuda_stream)
{
    if (!plan) return fail(nullptr, PHPRNG_EINVAL, "phprng_plan_launch: plan is NULL");
    std::lock_guard<std::mutex> lk(plan->ctx->mu);
    CU(plan->ctx, cudaSetDevice(plan->ctx->device));
    return plan_launch_locked(plan, c_base, r_base, (cudaStream_t)cuda_stream);
}

PH_API int phprng_plan_launch_graph(phprng_plan *plan, void *c_base, double *r_base,
                                    void *cuda_stream)
{
    if (!plan) return fail(nullptr, PHPRNG_EINVAL, "phprng_plan_launch_graph: plan is NULL");
    phprng_ctx *c = plan->ctx;
    std::lock_guard<std::mutex> lk(c->mu);
    CU(c, cudaSetDevice(c->device));
    if (!plan->gexec || plan->g_c != c_base || plan->g_r != r_base) {
        if (plan->gexec) {
            cudaGraphExecDestroy(plan->gexec);
            plan->gexec = nullptr;
        }
        if (!plan->cap_stream)
            CU(c, cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking));
        CU(c, cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = plan_launch_locked(plan, c_base, r_base, plan->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(plan->cap_stream, &g);
        if (rc != PHPRNG_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "phprng_plan_launch_graph: capture");
        e = cudaGraphInstantiate(&plan->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            plan->gexec = nullptr;
            return cuda_fail(c, e, "phprng_plan_launch_graph: instantiate");
        }
        plan->g_c = c_base;
        plan->g_r = r_base;
    }
    CU(c, cudaGraphLaunch(plan->gexec, (cudaStream_t)cuda_stream));
    for (const auto &fp : plan->final_pos) c->pos_host[fp.first] = fp.second;
    return PHPRNG_OK;
}

PH_API int phprng_plan_autotune(phprng_plan *plan, void *c_base, double *r_base,
                                phprng_tuning *best, void *cuda_stream)
{
    if (!plan) return fail(nullptr, PHPRNG_EINVAL, "phprng_plan_autotune: plan is NULL");
    phprng_ctx *c = plan->ctx;
    std::lock_guard<std::mutex> lk(c->mu);
    CU(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const uint32_t tiles[] = {4096, 16384, 65536};
    const int npts[] = {8, 4};
    cudaEvent_t e0, e1;
    CU(c, cudaEventCreate(&e0));
    CU(c, cudaEventCreate(&e1));
    phprng_tuning bestt = plan->tune;
    bestt.ms = -1.f;
    int rc = PHPRNG_OK;
    for (uint32_t tile : tiles) {
        rc = build_tiles(plan, tile);
        if (rc != PHPRNG_OK) break;
        for (int npt : npts) {
            const int maxb = batch_max_blocks_per_sm(npt, c->width != 32);
            for (int b = 1; b <= maxb && rc == PHPRNG_OK; ++b) {
                plan->tune.npt = npt;
                plan->tune.blocks_per_sm = b;
                rc = plan_launch_locked(plan, c_base, r_base, s);           // warm-up
                if (rc != PHPRNG_OK) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 2 && rc == PHPRNG_OK; ++r)
                    rc = plan_launch_locked(plan, c_base, r_base, s);
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) { rc = cuda_fail(c, e, "phprng_plan_autotune"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= 2.f;
                if (bestt.ms < 0.f || ms < bestt.ms) {
                    bestt = plan->tune;
                    bestt.ms = ms;
                }
            }
            if (rc != PHPRNG_OK) break;
        }
        if (rc != PHPRNG_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PHPRNG_OK) return rc;
    rc = build_tiles(plan, bestt.tile);
    if (rc != PHPRNG_OK) return rc;
    plan->tune = bestt;
    if (best) *best = bestt;
    return PHPRNG_OK;
}

PH_API int phprng_plan_tuning(const phprng_plan *plan, phprng_tuning *out)
{
    if (!plan || !out) return fail(nullptr, PHPRNG_EINVAL, "phprng_plan_tuning: NULL argument");
    *out = plan->tune;
    return PHPRNG_OK;
}

PH_API int phprng_plan_destroy(phprng_plan *plan)
{
    free_plan(plan);
    return PHPRNG_OK;
}

PH_API int phprng_generate_batch(phprng_ctx *ctx, const phprng_request *reqs, uint64_t nreq,
                                 void *c_base, double *r_base, void *cuda_stream)
{
    phprng_plan *pl = nullptr;
    int rc = phprng_plan_create(ctx, reqs, nreq, 0, &pl, cuda_stream);
    if (rc != PHPRNG_OK) return rc;
    rc = phprng_plan_launch(pl, c_base, r_base, cuda_stream);
    if (rc == PHPRNG_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "phprng_generate_batch");
    }
    free_plan(pl);
    return rc;
}
