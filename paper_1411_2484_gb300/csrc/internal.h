// internal.h -- data layout shared by the host layer, the C ABI and the
// kernels of libphprng (never installed, never seen by callers).
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <vector>

#include "../../include/phprng.h"
struct double2;   // vector_types.h (CUDA); pointers only here

#include "arith.cuh"

// Numbers per lane per warp group of the 32-bit and 64-bit generators (the
// unit of instruction-level parallelism of a lane; tuned on GB300: 8 and 4).
#ifndef PH_NPT32
#define PH_NPT32 8
#endif
#ifndef PH_NPT64
#define PH_NPT64 4
#endif

namespace phprng {

// One instance as the kernels read it: 64 bytes, read-only on the device.
// Derived on the host from {n, e} at creation.
struct alignas(16) DevInst {
    uint64_t n;      // prime modulus (Eq. 1)
    uint64_t ninv;   // 32-bit path: n^-1 mod 2^32, and K n^-1 mod 2^32 in the upper word
                     // (the exit product's constant, mont32c); 64-bit path: n^-1 mod 2^64
    uint64_t K;      // Montgomery exit constant R^(1-alpha) mod n, see mont_exit_constant()
    uint64_t e;      // exponent (its sliding-window program is a separate ExpProg)
    uint64_t V;      // floor(2^84 / yN): reciprocal for the integer-built R (32-bit path)
    uint32_t yN;     // (n+1) << (32 - bitlen(n+1)), normalised divisor (32-bit path)
    uint32_t ybits;  // bitlen(n+1)
    uint32_t fermat; // t when e = 2^t + 1 (straight chain of t squarings and one product), else 0
    uint32_t wide;   // 0: 32-bit path, 1: 64-bit path
    uint64_t aux;    // 64-bit path: 2^128 mod n, so x*y mod n = mont64(mont64(x, y), aux);
                     // 32-bit path: floor((2^95 - 1) / yN), the reciprocal of real32_fast
};
static_assert(sizeof(DevInst) == 64, "DevInst is one 64-byte line");

// Skip-generator constants for one (p, a) and one numbers-per-lane count
// NPT; passed to kernels by value.  Values in Montgomery form carry a
// factor 2^32 so that mont32(s, xM) = s*x mod p with s in plain form.
struct SkipConst {
    uint32_t p, pinv;      // p, p^-1 mod 2^32
    uint32_t aM;           // a * 2^32 mod p                      (one step, Eq. 9a)
    uint32_t aGM;          // a^(32*NPT) * 2^32 mod p             (one warp group)
    uint32_t aMq, aGMq;    // aM p^-1, aGM p^-1 mod 2^32 (constant products, mont32c)
    uint32_t lane[32];     // a^(NPT*j) * 2^32 mod p, j = lane    (lane start)
};

// The same for a wide skip prime p < 2^63 (64-bit moduli only): Montgomery
// products modulo p with R = 2^64, values in Montgomery form carrying 2^64.
struct SkipConst64 {
    uint64_t p, pinv;      // p, p^-1 mod 2^64
    uint64_t aM;           // a * 2^64 mod p                      (one step, Eq. 9a)
    uint64_t aGM;          // a^(32*NPT) * 2^64 mod p             (one warp group)
    uint64_t oneM;         // 2^64 mod p (1 in Montgomery form)
    uint64_t lane[32];     // a^(NPT*j) * 2^64 mod p, j = lane    (lane start)
};

// Generator state, structure of arrays in device memory, one entry per
// instance: the message m, the skip s, the last ciphertext c (the three
// values of the seven-integer state that change) and the stream position.
struct DevState {
    uint64_t *m, *s, *c, *pos;
};

// Arguments of one generate launch over instances [first, first+num).
// Split launch, for calls with too few instances to fill the GPU: every
// instance is cut into K chunks of Lc numbers (the last chunk shorter, or
// empty), and warp w runs chunk w % K of instance slot w / K.  A pre-pass
// (chunk_sums_kernel) leaves per slot q, at scratch[q*(K+1)]: the start
// message, the start skip, and the skip sums mod n of chunks 0 .. K-2; chunk
// c then starts from message m + (sums of chunks before it) and skip
// s a^(c Lc) (Eq. 6 over chunks).  K = 1 is the plain launch.
struct SplitArgs {
    uint32_t K = 1;                    // chunks per instance (num K < 2^32 when K > 1)
    uint64_t Kinv = 0;                 // ceil(2^64 / K) when K > 1
    uint64_t Lc = 0;                   // a multiple of 256
    uint32_t aLcM = 0;                 // a^Lc * 2^32 mod p
    uint32_t oneM = 0;                 // 2^32 mod p
    const uint64_t *scratch = nullptr;
};

struct GenArgs {
    const DevInst *inst;
    const ExpProg *prog;    // per-instance exponent programs
    const ExpProg8 *prog8 = nullptr;   // the 32-bit kernels' programs (tables of up to kProg8MaxTable odd powers)
    DevState st;
    SkipConst sk;
    uint64_t first, num, per_inst;
    void *c_out;            // uint32_t* (c_is_64 = 0) or uint64_t* (c_is_64 = 1), nullable
    double *r_out;          // nullable
    phprng_stats *stats;    // nullable
    uint32_t *edge;         // statistics scratch: gen32_edge_words(num, per_inst) words
    int c_is_64;
    int vec_ok;             // outputs allow 16-byte vector stores
    // nullable: warp w of the launch runs instance first + order[w] (a
    // permutation of 0 .. num-1, heaviest programs first); NULL = identity.
    // With statistics (whose pairs need adjacent instances) it orders the
    // blocks instead: block b of the launch runs logical block order[b].
    const uint32_t *order = nullptr;
    SplitArgs sp;                      // K = 1: no split
    int light = 0;                     // short exponent programs: the LIGHT instantiation
    // a wide skip prime (p >= 2^32, 64-bit moduli): the 64-bit generator
    // steps its skips with skw instead of sk (never split)
    int wide_skip = 0;
    SkipConst64 skw{};
};

// Exact prefix table of the skip generator's cycle (Eq. 7): with
// Pref(t) = sum_{i=1..t} (a^i mod p), the table holds T[j] = Pref(j*B) and
// the checkpoint powers P[j] = a^(j*B) mod p for j = 0 .. (p-1)/B.  Built on
// the device, shared by every instance (one (p, a) per context).
static constexpr uint32_t kSkipLog2B = 10;
static constexpr uint32_t kSkipB = 1u << kSkipLog2B;

// kind 0: a primitive root mod p (the pseudorandom skip, Eq. 5) with the
// prefix table; kind 1: a = 1, the constant skip s_k = s0 = b of Eq. 3 (b = 1
// is the unit skip), where a skip of k adds k b to the message and the per-
// instance array that holds cycle positions for kind 0 holds b instead.
struct SkipTable {
    uint32_t kind;         // 0 prefix table, 1 constant skip
    const uint64_t *T;     // prefix sums (exact, < 2^64 because p < 2^32)
    const uint32_t *P;     // checkpoint powers
    uint64_t nT;           // entries: (p-1)/B + 1
    uint64_t half;         // p(p-1)/2 = Pref(p-1), the sum over one cycle
    uint32_t p, pinv;      // p, p^-1 mod 2^32
    uint32_t aM;           // a * 2^32 mod p
    uint32_t oneM;         // 2^32 mod p (1 in Montgomery form)
    uint32_t laneM[32];    // a^(32*l) * 2^32 mod p: start of lane l's share of a tail
};

// One skip request after merging duplicates: advance instance `inst` by k.
struct SkipReq {
    uint64_t inst, k;
    uint64_t back;          // 0: forward by k; 1: backward by k (k <= position)
};

// ---- batched persistent launch (batch.cu) ----------------------------------
// One tile: `len` consecutive numbers of one instance starting after stream
// position `start`, written at element offsets c_off / r_off of the outputs.
static constexpr uint32_t kTileInstMask = 0x3fffffffu;   // instance index
static constexpr uint32_t kTileWide = 0x40000000u;       // 64-bit path
static constexpr uint32_t kTileWriteBack = 0x80000000u;  // ends the instance's last request
struct Tile {
    uint32_t inst;
    uint32_t len;
    uint64_t start, c_off, r_off;
};
static_assert(sizeof(Tile) == 32, "Tile is 32 bytes");

struct BatchArgs {
    const DevInst *inst;
    const ExpProg *prog;
    const ExpProg8 *prog8;          // 32-bit instances' exact-search programs
    DevState st;
    const uint64_t *m0, *L0;        // seed message and the seed skip's cycle position
    SkipTable tb;
    SkipConst sk32_8, sk32_4, sk64; // lane constants for NPT = 8, 4 (32-bit), PH_NPT64 (64-bit)
    const Tile *tiles;
    uint64_t ntiles;
    unsigned long long *counter;    // tile queue head, zeroed before each launch
    void *c_base;
    double *r_base;
    int c_is_64;
    int vec_ok;                     // c_base / r_base are 16-byte aligned
};
int launch_batch(const BatchArgs &a, int npt32, int blocks_per_sm, void *stream, std::string *err);
int batch_max_blocks_per_sm(int npt32, int c_is_64);

// ---- kernel launchers (gen.cu) -------------------------------------------
int gen_npt(int wide);   // numbers per lane per warp group of the 32/64-bit launch
int launch_gen32(const GenArgs &a, void *stream, std::string *err);
uint64_t gen32_edge_words(uint64_t num, uint64_t per_inst);
uint32_t gen32_stats_block_warps();   // instances per block of a statistics launch
uint64_t gen32_fixed_edge_words();
int launch_gen32_stats_fixed(const GenArgs &a, int dev, void *stream, std::string *err);
int launch_gen64(const GenArgs &a, void *stream, std::string *err);
// Serial-test consumer (serial.cu): D-tuples of floor(B R) bins of the
// launch's 32-bit streams added to hist[B^D]; D = 0: the poker test (hands of
// five floor(10 R) cards into hist[7]); sk for NPT 8.
int launch_serial(const GenArgs &a, int D, uint32_t B, unsigned long long *hist, void *stream,
                  std::string *err);
// Runs-test consumer (serial.cu): completed runs of R <= 1/2 and R > 1/2 by
// length (capped at lmax <= 64) added to hist[2 lmax]; sk for NPT 8.
int launch_runs(const GenArgs &a, int lmax, unsigned long long *hist, void *stream, std::string *err);
// Full-period pattern of the constant-skip generator (pattern.cu): P, pg for
// e and Pd, pgd for d = e^-1 mod n-1; one point per c0 in [c_lo, c_lo+L0).
// L1 = 0: cells of ceil(n / nb) over the whole range; L1 >= 1: cells of L1,
// tuples with a successor at or above nb L1 left out (a region near the origin).
int launch_pattern_const(const DevInst &P, const ExpProg &pg, const DevInst &Pd, const ExpProg &pgd,
                         uint32_t b, uint64_t c_lo, uint64_t L0, int D, uint32_t nb, uint32_t L1,
                         uint64_t *hist, void *stream, std::string *err);
// Fourier test (fourier.cu).  Twiddle tables for sequences of M = 2^lgM
// numbers: fourier_twiddle_count(lgM) double2, filled by launch_twiddles.
// launch_fourier: for nseq sequences of M doubles R (contiguous), the
// coefficients k < M/2 of the positive-exponent transform of R - 1/2 times
// scale2 = 1/(2 sqrt M) twice over (the real-input split halves), real and
// imaginary parts binned into hist[nbins] over [-w, w) (clamped); Z scratch of
// nseq M/2 double2; coef (nullable) gets nseq M/2 double2.
uint64_t fourier_twiddle_count(uint32_t lgM);
int launch_twiddles(double2 *tw, uint32_t lgM, double scale2, void *stream, std::string *err);
int launch_fourier(const double *R, uint64_t nseq, uint32_t lgM, const double2 *tw, double2 *Z,
                   uint32_t nbins, double w, double scale2, uint64_t *hist, double *coef, void *stream,
                   std::string *err);
// Interstream serial test (serial.cu): bins of a chunk c (Np streams x L
// numbers, instance-major) into binsT in interleaved order, then its
// D-tuples counted into hist (B^D counters).
static constexpr uint64_t kInterMaxChunk = 65535ull * 32;   // numbers per stream and chunk
// launch_inter_consts: per-stream bin constants k (Np x 16 bytes) of a call,
// before the chunks; launch_interstream then reads them.
int launch_inter_consts(const DevInst *inst, uint64_t first, uint64_t Np, uint32_t B, void *k, void *stream,
                        std::string *err);
// Interstream serial test for 2 <= D <= 8 (D dividing the number of 32-bit
// streams, B <= 2^16), fused: adjacent warps generate the D streams of a tuple
// group and count its tuples at once (group_order: group slots heaviest
// first, or NULL).
int launch_inter_groups(const GenArgs &a, int D, uint32_t B, unsigned long long *hist,
                        const uint32_t *group_order, void *stream, std::string *err);
int launch_interstream(const void *k, uint64_t Np, uint64_t L, const void *c, int c64,
                       int D, uint32_t B, uint32_t *binsT, unsigned long long *hist, void *stream,
                       std::string *err);
// Collision-test consumer (serial.cu): segments of S numbers into B bins,
// collision counts into hist[H]; `bins` is scratch for `cap` 32-bit bins
// (cap >= S): the streams' bins are written there in pieces of at most cap
// numbers and counted per segment before the next piece.
static constexpr uint64_t kCollBinsCap = 1ull << 28;
int launch_collision(const GenArgs &a, uint32_t S, uint32_t B, uint32_t H, unsigned long long *hist,
                     uint32_t *bins, uint64_t cap, void *stream, std::string *err);
// Full-period pattern by enumeration (pattern.cu): mtab[q] = (c_lo+q)^d mod n
// for q < L0, sk for NPT 8; hist has nb^(D-1) uint64 counters.
int launch_pattern(const DevInst &P, const ExpProg &pg, const SkipConst &sk, const uint32_t *mtab,
                   uint64_t L0, int D, uint32_t nb, uint32_t L1, uint64_t *hist, void *stream,
                   std::string *err);   // L1 as for launch_pattern_const
// Split launches: the pre-pass (sk8 = the NPT 8 skip constants) and the
// number of warps the 32-bit generator keeps resident on the current device.
int launch_chunk_sums(const GenArgs &a, const SkipConst &sk8, void *stream, std::string *err);
uint64_t gen_resident_warps();

// ---- skip-ahead (skip.cu) ------------------------------------------------
SkipTable derive_skip_table(uint64_t p, uint64_t a);   // constants; T, P set by the caller
int launch_build_skip_table(uint64_t p, uint64_t a, uint64_t *T, uint32_t *P, uint64_t *seg,
                            void *stream, std::string *err);
int launch_skip(const DevInst *inst, const ExpProg *prog, DevState st, const uint64_t *L0,
                SkipTable tbl, const SkipReq *reqs, uint64_t cnt, void *stream, std::string *err);

// Wide skip primes (p >= 2^32): Eq. 7 with the window sum formed by parallel
// stepping (no prefix table: the cycle has p - 1 > 2^32 terms).  One request
// advances instance `inst` by k (or goes back by k), using `scratch` (at least
// 1 + kWideSkipBlocks uint64 words, device memory) for the partial sums.
// The request is cut into pieces of at most kWideSkipPiece steps (one short
// launch sequence each); q = floor(k/(p-1)) full cycles add q p(p-1)/2 in
// closed form (Eq. 7), so only r = k mod (p-1) steps are formed.
static constexpr uint32_t kWideSkipBlocks = 1024;
static constexpr uint64_t kWideSkipPiece = 1ull << 34;
int launch_skip_wide(const DevInst *inst, const ExpProg *prog, DevState st, const SkipConst64 &skw,
                     uint64_t ainvM, const SkipReq &req, uint64_t *scratch, void *stream, std::string *err);

// ---- measurement (microbench.cu) ------------------------------------------
int run_microbench(int which, double *ops_per_s, void *stream, std::string *err);

// ---- host number theory (hostnt.cpp) -------------------------------------
uint64_t mulmod(uint64_t x, uint64_t y, uint64_t n);
uint64_t powmod(uint64_t b, uint64_t e, uint64_t n);
uint64_t gcd64(uint64_t a, uint64_t b);
bool is_prime(uint64_t n);
int bitlen(uint64_t x);
uint64_t inv_mod_2_64(uint64_t odd);
std::vector<uint64_t> prime_factors(uint64_t x);
bool is_primitive_root(uint64_t a, uint64_t p);
bool discrete_log(uint64_t p, uint64_t a, uint64_t s, uint64_t *L);
bool discrete_logs(uint64_t p, uint64_t a, const uint64_t *s, uint64_t count, uint64_t *L);
uint64_t mont_exit_constant(uint64_t n, const ExpProg &pg, int rbits);
DevInst derive_inst(const phprng_instance &in, int wide, ExpProg *prog);
int program_products(const ExpProg &pg);   // Montgomery products of one run, K included
// The 32-bit kernels' program of exponent e for the 32-bit prime n (products
// minimised over table sizes 1..kProg8MaxTable), with its exit constant.
ExpProg8 derive_prog8(uint64_t n, uint64_t e);
int program8_products(const ExpProg8 &pg);   // Montgomery products of one run, K included
SkipConst derive_skip(uint64_t p, uint64_t a, int npt);
SkipConst64 derive_skip64(uint64_t p, uint64_t a, int npt);
int validate_one(int width, const phprng_instance &in, uint32_t flags, std::string *msg);
int validate_all(int width, const phprng_instance *inst, uint64_t count, uint32_t flags,
                 uint64_t *bad, std::string *msg);
int draw_instances(int width, uint64_t count, uint64_t seed, uint32_t flags,
                   phprng_instance *out, std::string *msg);

}  // namespace phprng
