// serve.cpp -- the serving loop: continuous batching of generation requests
// over every stream of a context, kept in device memory.
//
// Requests (stream, length) arrive through phprng_server_submit, now or at a
// given future time (an open-loop arrival schedule is replayed exactly).  A
// scheduler thread:
//   admits arrived requests in FIFO order while their output fits in the
//     output arena (the admission bound), fixing each request's start
//     position on its stream (requests of one stream follow each other);
//   launches, whenever one of `inflight` CUDA streams is free, one batched
//     persistent launch (batch.cu) for everything admitted and not yet
//     launched -- so requests that arrive while others run are batched into
//     the next launch and overlap them on the device;
//   polls the launches' events and hands each finished request back with its
//     arrival and completion times (phprng_server_poll).
// Tiles derive their start state from the stream's seed (Eq. 7), so launches
// in flight at the same time never depend on each other; the streams' stored
// states are brought to their final positions when the server is destroyed.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <queue>
#include <thread>
#include <unordered_map>

#include "ctx.h"

using namespace phprng;

PH_API int64_t phprng_clock_ns(void)
{
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (int64_t)t.tv_sec * 1000000000ll + t.tv_nsec;
}

namespace {

struct Req {
    uint64_t id, tag, inst, len, start, off, bytes;
    int64_t arrival, done;
};

struct LaterArrival {
    bool operator()(const Req &a, const Req &b) const
    {
        return a.arrival != b.arrival ? a.arrival > b.arrival : a.id > b.id;
    }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Tile *h_tiles = nullptr;                    // pinned
    Tile *d_tiles = nullptr;
    unsigned long long *d_counter = nullptr;
    std::vector<Req> reqs;
    bool busy = false;
};

const uint64_t kSlotTiles = 1u << 16;           // tiles per launch
const uint64_t kAlign = 256;                    // arena slice alignment (bytes)

}  // namespace

struct phprng_server {
    phprng_ctx *ctx = nullptr;
    phprng_server_config cfg{};
    bool auto_tile = false;                      // cfg.tile was 0: tiles sized per launch
    uint64_t resident_warps = 1;                 // warps of batch_kernel the GPU keeps resident
    char *arena = nullptr;
    uint64_t arena_bytes = 0;
    std::map<uint64_t, uint64_t> free_list;     // offset -> size
    uint64_t outstanding = 0;
    std::vector<uint64_t> cursor;               // next start position per stream
    std::vector<uint64_t> pos_at_start;
    std::priority_queue<Req, std::vector<Req>, LaterArrival> future;
    std::deque<Req> waiting, pending;
    std::vector<Slot> slots;
    std::deque<phprng_completion> done;
    std::unordered_map<uint64_t, Req> live;     // completed, output not yet released
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::thread th;
    std::atomic<bool> stop{false};
    uint64_t next_id = 1;
    phprng_server_stats st{};
    int err_code = PHPRNG_OK;
    std::string err;
    uint64_t csz = 4;                            // bytes per ciphertext when stored
};

static uint64_t slice_bytes(const phprng_server *s, uint64_t len)
{
    uint64_t b = len * 8 + (s->cfg.want_c ? len * s->csz : 0);
    return (b + kAlign - 1) / kAlign * kAlign;
}

static bool arena_alloc(phprng_server *s, uint64_t bytes, uint64_t *off)
{
    for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const uint64_t rest = it->second - bytes, at = it->first + bytes;
            s->free_list.erase(it);
            if (rest) s->free_list[at] = rest;
            s->outstanding += bytes;
            return true;
        }
    }
    return false;
}

static void arena_free(phprng_server *s, uint64_t off, uint64_t bytes)
{
    s->outstanding -= bytes;
    auto it = s->free_list.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != s->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_list.erase(nx);
    }
    if (it != s->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_list.erase(it);
        }
    }
}

static void set_error(phprng_server *s, int code, const std::string &m)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err_code == PHPRNG_OK) {
        s->err_code = code;
        s->err = m;
    }
    s->cv_done.notify_all();
}

// Cuts the slot's requests into tiles and launches them on the slot's stream.
static int launch_slot(phprng_server *s, Slot &sl)
{
    phprng_ctx *c = s->ctx;
    uint64_t nt = 0;
    uint64_t tile = s->cfg.tile;
    if (s->auto_tile) {
        // about one tile per resident warp: a lightly loaded server finishes a
        // launch in the time of one short tile; never more than kSlotTiles tiles
        uint64_t total = 0;
        for (const Req &r : sl.reqs) total += r.len;
        const uint64_t round = 256;
        uint64_t t = (total + s->resident_warps - 1) / s->resident_warps;
        t = std::min<uint64_t>(std::max<uint64_t>((t + round - 1) / round * round, round), 4096);
        const uint64_t cap_t = (total + (kSlotTiles - sl.reqs.size()) - 1) / (kSlotTiles - sl.reqs.size());
        tile = std::max(t, (cap_t + round - 1) / round * round);
    }
    for (const Req &r : sl.reqs) {
        const uint32_t wide = c->wide[r.inst] ? kTileWide : 0u;
        const uint64_t r_off = r.off / 8;
        const uint64_t c_off = (r.off + r.len * 8) / s->csz;
        for (uint64_t k = 0; k < r.len; k += tile) {
            Tile &t = sl.h_tiles[nt++];
            t.len = (uint32_t)std::min<uint64_t>(tile, r.len - k);
            t.inst = (uint32_t)r.inst | wide;
            t.start = r.start + k;
            t.r_off = r_off + k;
            t.c_off = c_off + k;
        }
    }
    cudaError_t e = cudaMemcpyAsync(sl.d_tiles, sl.h_tiles, nt * sizeof(Tile),
                                    cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) {
        set_error(s, PHPRNG_ECUDA, std::string("server tile upload: ") + cudaGetErrorString(e));
        return PHPRNG_ECUDA;
    }
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
    a.tiles = sl.d_tiles;
    a.ntiles = nt;
    a.counter = sl.d_counter;
    a.c_base = s->cfg.want_c ? (void *)s->arena : nullptr;
    a.r_base = (double *)s->arena;
    a.c_is_64 = c->width != 32;
    a.vec_ok = 1;
    std::string err;
    int rc = launch_batch(a, 8, 0, sl.stream, &err);
    if (rc == PHPRNG_OK) {
        e = cudaEventRecord(sl.ev, sl.stream);
        if (e != cudaSuccess) {
            rc = PHPRNG_ECUDA;
            err = std::string("server event: ") + cudaGetErrorString(e);
        }
    }
    if (rc != PHPRNG_OK) {
        set_error(s, rc, "server launch: " + err);
        return rc;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.batches += 1;
    s->st.tiles += nt;
    return PHPRNG_OK;
}

static void scheduler(phprng_server *s)
{
    cudaSetDevice(s->ctx->device);
    const uint64_t max_batch = s->cfg.max_batch;
    const uint64_t tile = s->cfg.tile;
    for (;;) {
        bool busy_any = false;
        // completions
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) {
                busy_any = true;
                continue;
            }
            if (q != cudaSuccess) {
                set_error(s, PHPRNG_ECUDA, std::string("server batch: ") + cudaGetErrorString(q));
                sl.busy = false;
                continue;
            }
            const int64_t now = phprng_clock_ns();
            std::lock_guard<std::mutex> lk(s->mu);
            for (Req &r : sl.reqs) {
                r.done = now;
                phprng_completion cpl;
                cpl.id = r.id;
                cpl.tag = r.tag;
                cpl.inst = r.inst;
                cpl.start = r.start;
                cpl.len = r.len;
                cpl.r = (const double *)(s->arena + r.off);
                cpl.c = s->cfg.want_c ? (const void *)(s->arena + r.off + r.len * 8) : nullptr;
                cpl.arrival_ns = r.arrival;
                cpl.done_ns = now;
                s->done.push_back(cpl);
                s->live.emplace(r.id, r);
                s->st.completed += 1;
                s->st.numbers += r.len;
            }
            sl.reqs.clear();
            sl.busy = false;
            s->cv_done.notify_all();
        }
        // arrivals, admission, batch formation
        Slot *free_slot = nullptr;
        for (Slot &sl : s->slots)
            if (!sl.busy) { free_slot = &sl; break; }
        int64_t next_arrival = -1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const int64_t now = phprng_clock_ns();
            while (!s->future.empty() && s->future.top().arrival <= now) {
                s->waiting.push_back(s->future.top());
                s->future.pop();
            }
            while (!s->waiting.empty()) {
                Req &r = s->waiting.front();
                uint64_t off;
                if (!arena_alloc(s, r.bytes, &off)) break;           // FIFO: wait for space
                r.off = off;
                r.start = s->cursor[r.inst];
                s->cursor[r.inst] += r.len;
                s->pending.push_back(r);
                s->waiting.pop_front();
                s->st.admitted += 1;
            }
            s->st.max_waiting = std::max<uint64_t>(s->st.max_waiting, s->waiting.size());
            if (free_slot && !s->pending.empty()) {
                uint64_t tiles = 0;
                while (!s->pending.empty() && free_slot->reqs.size() < max_batch) {
                    const Req &r = s->pending.front();
                    const uint64_t rt = (r.len + tile - 1) / tile;
                    if (tiles + rt > kSlotTiles && !free_slot->reqs.empty()) break;
                    tiles += rt;
                    free_slot->reqs.push_back(r);
                    s->pending.pop_front();
                }
            }
            if (!s->future.empty()) next_arrival = s->future.top().arrival;
            const bool launching = free_slot && !free_slot->reqs.empty();
            const bool can_progress = launching || busy_any || !s->pending.empty();
            if (!can_progress && s->stop.load() && s->future.empty() && s->waiting.empty()) break;
            if (!can_progress) {
                // nothing to run: sleep until the next arrival, a submit or a release
                const int64_t wait = next_arrival < 0 ? 2000000
                                                      : std::max<int64_t>(0, next_arrival - now);
                if (wait > 20000)
                    s->cv_work.wait_for(lk, std::chrono::nanoseconds(std::min<int64_t>(wait - 10000, 2000000)));
            }
        }
        if (free_slot && !free_slot->reqs.empty()) {
            if (launch_slot(s, *free_slot) == PHPRNG_OK) {
                free_slot->busy = true;
            } else {
                free_slot->reqs.clear();
            }
        }
    }
}

PH_API int phprng_server_create(phprng_ctx *ctx, const phprng_server_config *cfg,
                                phprng_server **out)
{
    if (!out) return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: out is NULL");
    *out = nullptr;
    if (!ctx || !cfg) return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serving) return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: context already served");
    if (ctx->wide_skip)
        return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: served tiles start by Eq. 7 from the prefix "
                                        "table, which a skip prime p >= 2^32 does not have");
    if (ctx->count > kTileInstMask)
        return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: more than 2^30 instances");
    phprng_server *s = new (std::nothrow) phprng_server;
    if (!s) return fail(ctx, PHPRNG_ENOMEM, "phprng_server_create: host allocation failed");
    s->ctx = ctx;
    s->cfg = *cfg;
    if (!s->cfg.max_batch) s->cfg.max_batch = 4096;
    if (!s->cfg.inflight) s->cfg.inflight = 2;
    s->auto_tile = s->cfg.tile == 0;              // 0: sized per launch (launch_slot)
    if (!s->cfg.tile) s->cfg.tile = 4096;         // the largest tile, for admission checks
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        const int b = batch_max_blocks_per_sm(8, ctx->width != 32);
        s->resident_warps = (uint64_t)(sms > 0 ? sms : 1) * (b > 0 ? b : 1) * 8;
    }
    if (s->cfg.tile > (1u << 24) || s->cfg.inflight > 16) {
        delete s;
        return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: tile or inflight out of range");
    }
    s->csz = ctx->width == 32 ? 4 : 8;
    s->arena_bytes = cfg->output_budget_bytes / kAlign * kAlign;
    if (s->arena_bytes < kAlign) {
        delete s;
        return fail(ctx, PHPRNG_EINVAL, "phprng_server_create: output budget below 256 bytes");
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    int rc = e == cudaSuccess ? ensure_skip(ctx, nullptr) : cuda_fail(ctx, e, "cudaSetDevice");
    if (rc != PHPRNG_OK) { delete s; return rc; }
    e = cudaMalloc(&s->arena, s->arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(ctx, PHPRNG_ENOMEM, "phprng_server_create: output arena allocation failed");
    }
    s->free_list[0] = s->arena_bytes;
    s->slots.resize(s->cfg.inflight);
    for (Slot &sl : s->slots) {
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_tiles, kSlotTiles * sizeof(Tile));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_tiles, kSlotTiles * sizeof(Tile));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_counter, sizeof(unsigned long long));
        if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
        for (Slot &sl : s->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.ev) cudaEventDestroy(sl.ev);
            cudaFreeHost(sl.h_tiles);
            cudaFree(sl.d_tiles);
            cudaFree(sl.d_counter);
        }
        cudaFree(s->arena);
        delete s;
        return cuda_fail(ctx, e, "phprng_server_create: slot set-up");
    }
    s->cursor = ctx->pos_host;
    s->pos_at_start = ctx->pos_host;
    ctx->serving = true;
    s->th = std::thread(scheduler, s);
    *out = s;
    return PHPRNG_OK;
}

PH_API int phprng_server_submit(phprng_server *s, const uint64_t *inst, const uint64_t *len,
                                const uint64_t *tag, const int64_t *arrival_ns, uint64_t count,
                                uint64_t *first_id)
{
    if (!s) return fail(nullptr, PHPRNG_EINVAL, "phprng_server_submit: server is NULL");
    if (count && (!inst || !len)) return fail(nullptr, PHPRNG_EINVAL, "phprng_server_submit: NULL arrays");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err_code != PHPRNG_OK) return fail(nullptr, s->err_code, s->err);
    const int64_t now = phprng_clock_ns();
    for (uint64_t j = 0; j < count; ++j) {
        if (inst[j] >= s->ctx->count || len[j] == 0 || len[j] > (1ull << 32) ||
            (len[j] + s->cfg.tile - 1) / s->cfg.tile > kSlotTiles)
            return fail(nullptr, PHPRNG_EINVAL,
                        "phprng_server_submit: request " + std::to_string(j) +
                            ": instance out of range, or length outside [1, min(2^32, 65536 tiles)]");
        if (slice_bytes(s, len[j]) > s->arena_bytes)
            return fail(nullptr, PHPRNG_EBUDGET,
                        "phprng_server_submit: request " + std::to_string(j) +
                            " needs more output memory than the whole budget");
    }
    if (first_id) *first_id = s->next_id;
    for (uint64_t j = 0; j < count; ++j) {
        Req r;
        r.id = s->next_id++;
        r.tag = tag ? tag[j] : r.id;
        r.inst = inst[j];
        r.len = len[j];
        r.start = 0;
        r.off = 0;
        r.bytes = slice_bytes(s, len[j]);
        r.arrival = arrival_ns ? arrival_ns[j] : now;
        r.done = 0;
        s->future.push(r);
        s->st.submitted += 1;
    }
    s->cv_work.notify_all();
    return PHPRNG_OK;
}

PH_API int phprng_server_poll(phprng_server *s, phprng_completion *out, uint64_t max,
                              uint64_t *count, int64_t timeout_ns)
{
    if (!s || !count) return fail(nullptr, PHPRNG_EINVAL, "phprng_server_poll: NULL argument");
    *count = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ns > 0 && s->err_code == PHPRNG_OK)
        s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns),
                            [&] { return !s->done.empty() || s->err_code != PHPRNG_OK; });
    if (s->err_code != PHPRNG_OK && s->done.empty()) return fail(nullptr, s->err_code, s->err);
    uint64_t n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *count = n;
    return PHPRNG_OK;
}

PH_API int phprng_server_release(phprng_server *s, const uint64_t *ids, uint64_t count)
{
    if (!s) return fail(nullptr, PHPRNG_EINVAL, "phprng_server_release: server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint64_t j = 0; j < count; ++j) {
        auto it = s->live.find(ids[j]);
        if (it == s->live.end())
            return fail(nullptr, PHPRNG_EINVAL, "phprng_server_release: unknown or released id");
        arena_free(s, it->second.off, it->second.bytes);
        s->live.erase(it);
    }
    s->cv_work.notify_all();
    return PHPRNG_OK;
}

PH_API int phprng_server_copy(phprng_server *s, uint64_t id, double *r_dst, void *c_dst)
{
    if (!s) return fail(nullptr, PHPRNG_EINVAL, "phprng_server_copy: server is NULL");
    Req r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->live.find(id);
        if (it == s->live.end())
            return fail(nullptr, PHPRNG_EINVAL, "phprng_server_copy: unknown or released id");
        r = it->second;
    }
    cudaSetDevice(s->ctx->device);
    cudaError_t e = cudaSuccess;
    if (r_dst) e = cudaMemcpy(r_dst, s->arena + r.off, r.len * 8, cudaMemcpyDefault);
    if (e == cudaSuccess && c_dst) {
        if (!s->cfg.want_c)
            return fail(nullptr, PHPRNG_EINVAL, "phprng_server_copy: server stores no ciphertexts");
        e = cudaMemcpy(c_dst, s->arena + r.off + r.len * 8, r.len * s->csz, cudaMemcpyDefault);
    }
    if (e != cudaSuccess) return fail(nullptr, PHPRNG_ECUDA, std::string("phprng_server_copy: ") + cudaGetErrorString(e));
    return PHPRNG_OK;
}

PH_API int phprng_server_stats_get(phprng_server *s, phprng_server_stats *out)
{
    if (!s || !out) return fail(nullptr, PHPRNG_EINVAL, "phprng_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->outstanding_bytes = s->outstanding;
    out->waiting = s->waiting.size() + s->future.size();
    return PHPRNG_OK;
}

PH_API int phprng_server_destroy(phprng_server *s)
{
    if (!s) return PHPRNG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
        // requests not yet arrived are dropped; admitted ones finish
        while (!s->future.empty()) s->future.pop();
        s->waiting.clear();
        s->cv_work.notify_all();
    }
    s->th.join();
    phprng_ctx *c = s->ctx;
    int rc = s->err_code;
    cudaDeviceSynchronize();
    // bring the stored states to the served positions (Eq. 7 skip kernel)
    std::vector<SkipReq> reqs;
    for (uint64_t i = 0; i < c->count; ++i)
        if (s->cursor[i] != s->pos_at_start[i]) reqs.push_back({i, s->cursor[i] - s->pos_at_start[i], 0});
    std::string err;
    if (!reqs.empty() && rc == PHPRNG_OK) {
        SkipReq *d = nullptr;
        cudaError_t e = cudaMalloc(&d, reqs.size() * sizeof(SkipReq));
        if (e == cudaSuccess)
            e = cudaMemcpy(d, reqs.data(), reqs.size() * sizeof(SkipReq), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            rc = launch_skip(c->d_inst, c->d_prog, c->st, c->d_L0, c->tbl, d, reqs.size(), nullptr, &err);
            e = cudaDeviceSynchronize();
        }
        cudaFree(d);
        if (e != cudaSuccess && rc == PHPRNG_OK) {
            rc = PHPRNG_ECUDA;
            err = cudaGetErrorString(e);
        }
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (rc == PHPRNG_OK) c->pos_host = s->cursor;
        c->serving = false;
    }
    for (Slot &sl : s->slots) {
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.ev);
        cudaFreeHost(sl.h_tiles);
        cudaFree(sl.d_tiles);
        cudaFree(sl.d_counter);
    }
    cudaFree(s->arena);
    std::string msg = s->err.empty() ? err : s->err;
    delete s;
    if (rc != PHPRNG_OK) return fail(c, rc, "phprng_server_destroy: " + msg);
    return PHPRNG_OK;
}
