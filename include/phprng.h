/*
 * phprng.h -- C ABI of the GB300 (sm_103a) Pohlig-Hellman exponentiation-
 * cipher pseudorandom generator.
 *
 * Method: P. D. Beale, "A new class of scalable parallel pseudorandom number
 * generators based on Pohlig-Hellman exponentiation ciphers", arXiv:1411.2484.
 * Every instance owns a prime modulus n and an exponent e with
 * gcd(e, n-1) = 1 (Eq. 1) and a prime-modulus skip generator (p, a) with
 * p < n and a a primitive root mod p (Eq. 5).  Its state is the seven
 * integers {m, s, c, n, e, p, a} ("Message skipping algorithms"), of which
 * m, s and c change.  One number is one pass of the implementation algorithm
 * (Eq. 9):
 *     s := a s mod p;  m := (m + s) mod n;  c := m^e mod n;  R := (c+1)/(n+1).
 *
 * Conventions shared by every entry point:
 *  - Every function returns a phprng_status and never throws or aborts.
 *    A call rejected by its argument checks leaves the context unchanged;
 *    calls that work in chunks (phprng_fourier_test,
 *    phprng_interstream_serial_test) and fail on the device part-way leave
 *    the streams advanced by the chunks completed, as phprng_get_state
 *    reports.  phprng_last_error() gives a one-line message.
 *  - Instance numbers are 0-based indexes into the table given at creation.
 *  - The stream position t of an instance counts the numbers produced so far.
 *    Output j (0-based) of a call is number t+j+1 of the stream, c_{t+j+1}:
 *    the first number ever produced comes from (m0, s0) by Eq. 9a-9c.
 *  - Device work is enqueued on the caller's CUDA stream (a cudaStream_t
 *    passed as void*, NULL = legacy default stream) and is asynchronous,
 *    unless an output pointer is host memory (see phprng_generate).
 *  - The library owns the instance table, the generator state and the skip
 *    table in device memory.  The caller owns every output buffer.
 *  - Widths: 32 = moduli below 2^32 (c is uint32_t), 64 = moduli below 2^64
 *    (c is uint64_t), 0 = mixed table, each instance on the 32-bit path when
 *    n < 2^32 and on the 64-bit path otherwise (c is uint64_t).
 */
#ifndef PHPRNG_H
#define PHPRNG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
    PHPRNG_OK = 0,
    PHPRNG_EINVAL = 1,      /* bad argument: null or misaligned pointer, range, size, width */
    PHPRNG_ENOTPRIME = 2,   /* n (or (n-1)/2 when a safe prime is required) is composite */
    PHPRNG_EEXPONENT = 3,   /* e outside [3, n-2] or gcd(e, n-1) != 1 (Eq. 1, Eq. 2) */
    PHPRNG_ESKIP = 4,       /* (p, a, s0) is not a valid skip generator (Eq. 5) */
    PHPRNG_EDUPLICATE = 5,  /* two instances share a modulus (parameter splitting) */
    PHPRNG_ENOMEM = 6,      /* host or device allocation failed */
    PHPRNG_ECUDA = 7,       /* a CUDA runtime call failed; the message names it */
    PHPRNG_ETIMEOUT = 8,    /* a bounded device or host wait ran out */
    PHPRNG_EBUDGET = 9      /* admission refused: the output-byte budget is full */
} phprng_status;

/* Creation flags. */
#define PHPRNG_REQUIRE_SAFE_PRIME 0x1u  /* (n-1)/2 must be prime (Implementation section) */
#define PHPRNG_ALLOW_SHARED_N     0x2u  /* allow two instances with the same n */

/* One instance as the caller describes it (caller-owned input).
 * n  prime modulus, 5 <= n < 2^32 (width 32) or < 2^64 (width 64, 0)
 * e  exponent, 3 <= e <= n-2, gcd(e, n-1) = 1
 * p  skip-generator prime, 3 <= p < n, p < 2^32; the same (p, a) for every
 *    instance of a context.  For 64-bit moduli p may reach 2^63 (the
 *    Implementation section's wide skip generator, period n(p-1) up to
 *    2^127); a is then checked with the factors of p-1 found by Pollard's
 *    rho, skip-ahead forms its window sum by parallel stepping (at most 2^40
 *    steps beyond whole cycles per call), and batched requests and the
 *    server are not available (their tiles start from the prefix table)
 * a  primitive root mod p (the pseudorandom skip s_k = a s_(k-1) mod p, Eq. 5),
 *    or a = 1 for the constant skip s_k = s0 = b of "Message skipping
 *    algorithms" (Eq. 3; b = 1 is the unit skip, the cipher in counter mode,
 *    with period n): then p is any prime with 2 <= p < n, p < 2^32 (p = 2 with
 *    s0 = 1 gives the unit skip), and a skip by k adds k b to the message
 * m0 initial message, 0 <= m0 < n
 * s0 initial skip, 1 <= s0 <= p-1 */
typedef struct {
    uint64_t n, e, p, a, m0, s0;
} phprng_instance;

/* Per-stream statistics of one generate call (fused consumer mode; 32-bit
 * moduli).  N = numbers of the call for this stream, c_k its ciphertexts,
 * R_k = (c_k+1)/(n+1) as in Eq. 9d.  All sums are exact integers:
 *   x = sum (c_k+1),  y = sum (c_k+1)^2,
 *   z = sum (c_k+1)(c'_k+1) with c' the next instance of the call (stream
 *       alpha+1 in the interstream ordering of "Message skipping
 *       algorithms", last item); 0 for the last instance of the call,
 *   hist[b] = #{k : floor(256 R_k) = b}.
 * Doubles: mean = RN(RN(x) / RN(N(n+1))),
 *          var  = RN(RN(N y - x^2) / RN(N(N-1)(n+1)^2))   (0 when N < 2),
 *          corr = RN(RN(z) / RN(N(n+1)(n'+1)))             (0 for the last).
 * Integers of 128 bits are stored as {lo, hi}. */
typedef struct {
    uint64_t x_lo, x_hi;
    uint64_t y_lo, y_hi;
    uint64_t z_lo, z_hi;
    uint64_t count;
    double mean, var, corr;
    uint32_t hist[256];
} phprng_stats;

typedef struct phprng_ctx phprng_ctx;   /* opaque, library-owned */

/* ---------------------------------------------------------------- lifetime */

/* Validates `count` instances on the host and uploads them to the current
 * CUDA device.  Validation (Implementation section): n prime by trial
 * division by the primes below 256 and then the deterministic Rabin-Miller
 * test with bases 2,3,5,7,11 (n < 2^32) or the twelve primes up to 37
 * (n < 2^64); with PHPRNG_REQUIRE_SAFE_PRIME also (n-1)/2; e as above; p
 * prime and a a primitive root mod p (a^((p-1)/q) != 1 for every prime q
 * dividing p-1); moduli distinct unless PHPRNG_ALLOW_SHARED_N.
 * width: 32, 64 or 0 (mixed).  On success *out is a new context whose every
 * stream is at position 0.  On failure *out is NULL, nothing is allocated,
 * and phprng_last_error(NULL) names the first offending instance.
 * cuda_stream orders the uploads. */
int phprng_create(phprng_ctx **out, int width, const phprng_instance *inst,
                  uint64_t count, uint32_t flags, void *cuda_stream);

/* Draws `count` instances from a 64-bit seed with phprng_draw_instances()
 * and creates a context from them. */
int phprng_create_seeded(phprng_ctx **out, int width, uint64_t count, uint64_t seed,
                         uint32_t flags, void *cuda_stream);

/* Frees the context and its device memory after the device is idle with
 * respect to it (synchronizes the device).  NULL is accepted. */
int phprng_destroy(phprng_ctx *ctx);

/* Message of the last failed call on ctx, or of the calling thread's last
 * failed create when ctx is NULL.  Never NULL; owned by the library. */
const char *phprng_last_error(const phprng_ctx *ctx);

/* Static text for a status code. */
const char *phprng_status_string(int status);

/* ---------------------------------------------------------------- generation */

/* Produces per_inst consecutive numbers (Eq. 9) for each of the instances
 * first .. first+num_inst-1 and advances their streams by per_inst.
 * Outputs, instance-major (instance first+i, number j at index i*per_inst+j):
 *   c_out  ciphertexts c (uint32_t for width 32, uint64_t otherwise), or NULL
 *   r_out  R = (c+1)/(n+1) as IEEE double: for n < 2^32 the correctly
 *          rounded quotient; for 64-bit n, RN(RN(c+1)/RN(n+1)) -- or NULL
 *   stats_out  num_inst phprng_stats (32-bit instances only), or NULL.
 *          With c_out and r_out NULL this is the fused mode: nothing but the
 *          statistics is written.
 * Pointers may be device memory (asynchronous on cuda_stream) or host memory
 * (pinned or pageable; the call then stages through device buffers, copies
 * back, and returns after the data is on the host).  c_out/r_out must be
 * aligned to their element size.  per_inst = 0 is a no-op.
 * Work layout (results do not depend on it): a call of 1,024 instances or
 * more runs them heaviest exponent first; a call with too few instances to
 * fill the GPU cuts each instance's numbers into chunks (Eq. 6 over chunks:
 * a pre-pass kernel sums each chunk's skips) and then takes a stream-ordered
 * scratch of num_inst*(K+1) uint64 (K <= 4096 chunks) for the duration of
 * the call.  Calls on overlapping instance ranges must be ordered on the
 * device (they share the stored states). */
int phprng_generate(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                    void *c_out, double *r_out, phprng_stats *stats_out, void *cuda_stream);

/* The fused-statistics call of phprng_generate (c_out = r_out = NULL) for
 * callers that must not allocate GPU memory: a process whose caching
 * allocator already holds the device's memory, a latency-critical loop where
 * an allocation would synchronise the device, or code that may only allocate
 * at start-up.  The paper has no counterpart; it is a property of this
 * library.  It allocates and frees no device memory (nor host memory when it
 * succeeds): its only scratch, the ciphertext rows that pair instances
 * across thread blocks, lives in a fixed array of 2^20 uint32 words (4 MiB)
 * that every device holds while the library is loaded.  Limit:
 * 2 * ceil(num_inst/8) * per_inst <= 2^20, else PHPRNG_EINVAL naming the
 * limit.  stats_out must be device memory (num_inst phprng_stats).  The first
 * call on a device looks up the array's device address once and keeps it for
 * the rest of the process (make that first call before any CUDA stream
 * capture); the address belongs to the device's primary context, so the
 * library must not be used on a device after cudaDeviceReset there.  All calls share the array and
 * leave their rows in it; every row is fully written before it is read, so
 * nothing needs clearing, but calls that overlap on the GPU (unordered
 * streams) race on it.  Results, state updates and errors are otherwise
 * those of phprng_generate with stats_out. */
int phprng_generate_stats_noalloc(phprng_ctx *ctx, uint64_t first, uint64_t num_inst,
                                  uint64_t per_inst, phprng_stats *stats_out, void *cuda_stream);

/* Advances instance inst_ids[i] by k[i] positions without producing output,
 * by the closed form Eq. 7 (k = q(p-1) + r: s' = s a^r mod p and
 * m' = m + q p(p-1)/2 + sum_{j=1..r} (s a^j mod p) mod n), with the sum read
 * from an exact prefix-sum table of the skip cycle of (p, a) (built on the
 * device at the first call, then kept); for the constant skip (a = 1)
 * m' = m + k s mod n and s' = s (Eq. 3 with s_k = b), with no table.  inst_ids and k are host arrays of
 * cnt entries; an instance may appear more than once (the skips add). */
int phprng_skip(phprng_ctx *ctx, const uint64_t *inst_ids, const uint64_t *k, uint64_t cnt,
                void *cuda_stream);

/* Serial-test consumer (Tests section, items 1-5: the one-dimensional
 * frequency test and the two- to five-dimensional serial tests) for 32-bit
 * moduli.  Generates per_inst numbers of each instance first ..
 * first+num_inst-1 (advancing their streams exactly as phprng_generate does)
 * without storing them: each stream's numbers of this call, in order, form
 * consecutive non-overlapping D-tuples (R_{t+1}, ..., R_{t+D}) (a remainder of
 * fewer than D numbers at the end of the call is left out); coordinate d falls
 * in bin b_d = floor(B R), R the double of Eq. 9d and B R one IEEE double
 * product (truncated), and each tuple adds one to
 * hist[b_0 + B b_1 + ... + B^(D-1) b_(D-1)].  That bin equals the exact
 * floor(B (c+1)/(n+1)) except where (c+1)/(n+1) is exactly k/B and the double
 * product falls below k (B = 100: k = 29, 57, 58), where it is k - 1, as the
 * double arithmetic gives it.  hist: device memory,
 * B^D uint64 counters, added to (clear it first); all streams of the call
 * share it.  The paper's sizes: D = 1, B = 2^20; D = 2, B = 2^10; D = 3,
 * B = 100; D = 4, B = 32; D = 5, B = 16.  Limits: 1 <= D <= 8, B a power of
 * two up to 2^20 or any B up to 2^16, B^D <= 2^24; else PHPRNG_EINVAL.  The
 * chi-square against the uniform expectation is left to the caller.
 * Asynchronous on cuda_stream. */
int phprng_serial_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                       int D, uint32_t B, uint64_t *hist, void *cuda_stream);

/* Poker-test consumer (Tests section: five cards, ten denominations) for
 * 32-bit moduli.  Like phprng_serial_test with D = 5: each stream's numbers of
 * the call form consecutive non-overlapping hands of five; card k has
 * denomination floor(10 R_k); the hand adds one to hist[category], with
 * categories 0 all different, 1 one pair, 2 two pairs, 3 three of a kind,
 * 4 full house, 5 four of a kind, 6 five of a kind (exact probabilities
 * 0.3024, 0.504, 0.108, 0.072, 0.009, 0.0045, 0.0001).  hist: device memory,
 * 7 uint64 counters, added to.  Streams advance by per_inst.  Asynchronous on
 * cuda_stream. */
int phprng_poker_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                      uint64_t *hist, void *cuda_stream);

/* Collision-test consumer (Tests section: 2^14 numbers into 2^20 bins) for
 * 32-bit moduli.  Each stream's numbers of the call form consecutive
 * segments of S numbers (a remainder of fewer than S is left out); in a
 * segment, a number whose bin floor(B R) (the double product, as in
 * phprng_serial_test) already holds an earlier number of
 * the segment is a collision, and the segment's collision count C adds one to
 * hist[min(C, H-1)].  Expected count per segment S - B (1 - (1 - 1/B)^S)
 * (about 127.3 at the paper's S = 2^14, B = 2^20).  hist: device memory, H
 * uint64 counters, added to.  Limits: S a multiple of 256 from 256 to 2^24;
 * B a power of two up to 2^20 or any B up to 2^16; 1 <= H <= 2^16.  The
 * bins of the complete segments are written to a stream-ordered scratch of
 * 4 bytes per number, at most 2^28 numbers (1 GiB) at a time (larger calls
 * run in pieces), and each segment is counted in a B-bit bitmap in shared
 * memory.  Streams advance by per_inst.  Asynchronous on cuda_stream. */
int phprng_collision_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                          uint32_t S, uint32_t B, uint32_t H, uint64_t *hist, void *cuda_stream);

/* Runs-test consumer (Tests section: runs of 0's, R <= 1/2, and 1's,
 * R > 1/2) for 32-bit moduli.  Each stream's numbers of the call, in order,
 * give bits b_k = (R_k > 1/2); every maximal run of equal bits that ends before
 * the call's last number adds one to hist[b * lmax + min(L, lmax) - 1] (L its
 * length; the first run starts at the call's first number, the run still
 * open at the last number is left out).  For fair independent bits a
 * completed run has length L with probability 2^-L.  hist: device memory,
 * 2 lmax uint64 counters, added to; 1 <= lmax <= 64; per_inst < 2^32.
 * Streams advance by per_inst.  Asynchronous on cuda_stream. */
int phprng_runs_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                     int lmax, uint64_t *hist, void *cuda_stream);

/* Interstream serial test (Tests section, interstream correlations): the
 * per_inst numbers that each instance of [first, first + num_inst) draws in
 * this call (Eq. 9) are taken in the paper's interleaved order -- number 1 of
 * every instance in order, then number 2 of every instance, and so on -- and
 * that sequence of num_inst * per_inst numbers is cut into consecutive
 * non-overlapping D-tuples (the last num_inst * per_inst mod D numbers are left
 * out); each tuple adds one to hist[b_1 + B b_2 + ... + B^(D-1) b_D], b =
 * floor(B R) (the double product, as in phprng_serial_test).  Limits as
 * phprng_serial_test: 1 <= D <= 8, B a power of two up
 * to 2^20 or at most 2^16, B^D <= 2^24, 32-bit instances.  hist: device
 * memory, B^D uint64 counters, added to.  Streams advance by per_inst.
 * Asynchronous on cuda_stream.  In a 32-bit context D = 1 is the frequency
 * test's kernel, and D >= 2 dividing num_inst with B <= 2^16 takes no
 * scratch: the D streams of each tuple group run as D warps that count their
 * tuples as they generate them (only an order of the groups, num_inst / D
 * words, when there are many).  Otherwise a scratch of about 2^25 numbers
 * (ciphertexts and bins) from the stream-ordered allocator. */
int phprng_interstream_serial_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                                   int D, uint32_t B, uint64_t *hist, void *cuda_stream);

/* Fourier test (Tests section): every instance of [first, first + num_inst)
 * draws per_inst numbers R (Eq. 9), cut into per_inst / M consecutive
 * sequences of M = 2^log2M; for each sequence x_j = R_j - 1/2 and
 * xhat_k = M^(-1/2) sum_j x_j exp(+2 pi i j k / M), k = 0 .. M/2 - 1, and the
 * real and imaginary parts of every xhat_k each add one to
 * hist[floor((v + w) (nbins / 2w))], clamped to bins 0 and nbins - 1 outside
 * [-w, w).  For uniform R both parts are close to normal with variance 1/24
 * (k > 0).  Computed in FP64 on the device (the M real numbers as M/2 complex
 * points, a four-step FFT of those, and the split into the real transform),
 * so a coefficient differs from the plain sum by rounding (about 1e-15
 * relative); a part within that of a bin edge may fall in the neighbouring
 * bin.  coef_out (nullable, device, 16-byte aligned) receives the
 * coefficients as (re, im) pairs: sequence q of the call (instances in order,
 * their sequences in order) at coef_out[2 (q M/2 + k)].  Limits: 32-bit
 * instances, 2 <= log2M <= 20, per_inst a multiple of M, 1 <= nbins <= 2^24,
 * w > 0.  hist: device memory, nbins uint64 counters, added to.  Streams
 * advance by per_inst.  Asynchronous on cuda_stream (scratch comes from the
 * stream-ordered allocator: at most 2^26 numbers of R, as many bytes of
 * transform scratch, and about M twiddle factors). */
int phprng_fourier_test(phprng_ctx *ctx, uint64_t first, uint64_t num_inst, uint64_t per_inst,
                        uint32_t log2M, uint32_t nbins, double w, uint64_t *hist, double *coef_out,
                        void *cuda_stream);

/* Full-period D-dimensional pattern of one instance (32-bit n) by
 * enumeration, as the paper derives after Eq. 7: over the whole period
 * n(p-1) the value c0 occurs p-1 times, once with each next skip s in
 * (Z/pZ)*, always with message m = c0^d mod n (d = e^-1 mod n-1, Eq. 2), so
 * the tuples that start at c0 are c_(k+j) = (m + s + a s + ... + a^(j-1) s)^e
 * mod n (skip terms mod p, sums mod n), j = 1 .. D-1.  For every c0 in
 * [c_lo, c_lo + L0) and every s in 1 .. p-1 the point adds one to
 * hist[b_1 + nb b_2 + ... + nb^(D-2) b_(D-1)], b_j = floor(c_(k+j) / L1) with
 * L1 = ceil(n / nb): L0 (p-1) points and (D-1) L0 (p-1) exponentiations
 * instead of n(p-1) steps.  The paper's volumes: L0 = 2^7 and nb^(D-1) = 2^24
 * for D = 3, 4, 5 (expected count (p-1) L0 (L1/n)^(D-1) per volume).
 * inst: validated like one instance of phprng_create (width 32, no flags);
 * its m0 and s0 are not used.  Limits: 1 <= L0 <= 2^20, c_lo + L0 <= n,
 * 2 <= D <= 8, nb^(D-1) <= 2^24.  hist: device memory, nb^(D-1) uint64
 * counters, added to.  Needs no context; asynchronous on cuda_stream; errors
 * are reported through phprng_last_error(NULL). */
int phprng_pattern(const phprng_instance *inst, uint64_t c_lo, uint64_t L0, int D, uint32_t nb,
                   uint64_t *hist, void *cuda_stream);

/* Full-period D-dimensional pattern of the constant-skip generator of one
 * instance ("Message skipping algorithms": s_k = b, m_k = m_0 + k b mod n,
 * period n; b = 1 is the unit skip, encryption of a counter).  Each c0 occurs
 * once per period, with message m = c0^d mod n (d = e^-1 mod n-1, Eq. 2), and
 * the tuple that starts there continues with c_(k+j) = (m + j b)^e mod n: for
 * every c0 in [c_lo, c_lo + L0) the point adds one to hist[b_1 + nb b_2 + ...
 * + nb^(D-2) b_(D-1)], b_j = floor(c_(k+j) / L1), L1 = ceil(n / nb).  Uses n and
 * e of inst (validated as for phprng_create, width 32).  Limits: 1 <= b < n,
 * 1 <= L0, c_lo + L0 <= n (L0 = n, c_lo = 0 is the whole period), 2 <= D <= 8,
 * nb^(D-1) <= 2^24.  hist: device memory, nb^(D-1) uint64 counters, added to.
 * Asynchronous on cuda_stream; errors through phprng_last_error(NULL). */
int phprng_pattern_const(const phprng_instance *inst, uint64_t b, uint64_t c_lo, uint64_t L0, int D,
                         uint32_t nb, uint64_t *hist, void *cuda_stream);

/* The full-period patterns over a region near the origin, as the paper's
 * Figs. 2-4 show them (magnified squares and slabs): as phprng_pattern and
 * phprng_pattern_const, but the cells have the given width L1 >= 1 and only
 * the tuples whose successors all lie below nb L1 are counted, so that
 * hist[b_1 + nb b_2 + ...], b_j = floor(c_(k+j) / L1), covers the region
 * [0, nb L1)^(D-1) of the successors of the starting values c0 in
 * [c_lo, c_lo + L0).  With L1 = ceil(n / nb) they equal the whole-range calls.
 * Examples: Fig. 3's 2^7 x 2^7 square, one call per c0 in [0, 2^7) with
 * L0 = 1, D = 2, nb = 2^7, L1 = 1 (each pair appears once or not at all);
 * Fig. 4's slab 2^9 x 2^16 x 2^16 in 16 subslabs, c_lo = 0, L0 = 2^9, D = 3,
 * nb = 4, L1 = 2^14.  Limits and errors otherwise those of the whole-range
 * calls. */
int phprng_pattern_region(const phprng_instance *inst, uint64_t c_lo, uint64_t L0, int D, uint32_t nb,
                          uint32_t L1, uint64_t *hist, void *cuda_stream);
int phprng_pattern_const_region(const phprng_instance *inst, uint64_t b, uint64_t c_lo, uint64_t L0, int D,
                                uint32_t nb, uint32_t L1, uint64_t *hist, void *cuda_stream);

/* Moves instance inst_ids[i] to absolute stream position pos[i], forward or
 * backward: afterwards its next number is number pos[i]+1 of the stream
 * counted from its seed, and its state (m, s, c) is the one generation would
 * have left there (c = 0 at position 0).  Both directions use Eq. 7 with the
 * prefix table: backward by k from cycle position L, the earlier state sits at
 * L' = L - k mod (p-1), with s' = a^L' and m' = m - (q p(p-1)/2 +
 * sum_{j=1..r} a^(L'+j) mod p) mod n.  With phprng_get_state this saves and
 * restores streams (save the position, seek back to it later).  inst_ids and
 * pos are host arrays of cnt entries; when an instance appears more than once
 * its last entry counts.  Asynchronous on cuda_stream; builds the prefix table
 * at the first call as phprng_skip does. */
int phprng_seek(phprng_ctx *ctx, const uint64_t *inst_ids, const uint64_t *pos, uint64_t cnt,
                void *cuda_stream);

/* ---------------------------------------------------------------- batches */

/* One request of a batch: `len` consecutive numbers of instance `inst`,
 * starting after stream position `offset` (the request's first output is
 * number offset+1, reached by Eq. 7 without producing the numbers before it),
 * or, with offset = PHPRNG_CONTINUE, right after the instance's previous
 * request in the same batch (after its current position for the first one).
 * Outputs go to c_base[c_off + j] and r_base[r_off + j], j < len.  Requests
 * with len = 0 are ignored (they move no position). */
#define PHPRNG_CONTINUE UINT64_MAX
typedef struct {
    uint64_t inst, offset, len, c_off, r_off;
} phprng_request;

typedef struct phprng_plan phprng_plan;   /* opaque, library-owned */

/* Launch configuration of a plan: numbers per tile, numbers per lane per warp
 * group of the 32-bit path (4 or 8), resident blocks per SM (0 = as many as
 * fit), and the time the autotuner measured for it (ms, 0 if never timed). */
typedef struct {
    uint32_t tile;
    int32_t npt;
    int32_t blocks_per_sm;
    float ms;
} phprng_tuning;

/* Resolves a batch of requests into tiles of at most `tile` numbers (0 = a
 * default) and uploads them: the plan for one persistent launch that serves
 * every request, whatever its instance width, length and start.  Start
 * positions are fixed here (PHPRNG_CONTINUE is resolved against the context's
 * positions now).  After every launch of the plan, each instance it touches
 * is positioned at the end of its last request (in request order), with its
 * state written back.  Builds the skip table on first use.  The plan keeps a
 * pointer to ctx: destroy it before the context.  reqs is a host array. */
int phprng_plan_create(phprng_ctx *ctx, const phprng_request *reqs, uint64_t nreq,
                       uint32_t tile, phprng_plan **out, void *cuda_stream);

/* One persistent launch of the plan on cuda_stream (a memset of the tile
 * queue and one kernel; both may be captured in a CUDA graph).  c_base and
 * r_base are device memory (either may be NULL); the caller sizes them for
 * the largest c_off + len and r_off + len of the plan. */
int phprng_plan_launch(phprng_plan *plan, void *c_base, double *r_base, void *cuda_stream);

/* The same launch through a CUDA graph that the plan captures on first use
 * for these output pointers and replays afterwards. */
int phprng_plan_launch_graph(phprng_plan *plan, void *c_base, double *r_base, void *cuda_stream);

/* Times plan launches over tile sizes, numbers per lane and blocks per SM
 * (CUDA events on cuda_stream; the outputs are written each time with the
 * same values), keeps the fastest configuration in the plan and returns it. */
int phprng_plan_autotune(phprng_plan *plan, void *c_base, double *r_base,
                         phprng_tuning *best, void *cuda_stream);

/* Current configuration of the plan. */
int phprng_plan_tuning(const phprng_plan *plan, phprng_tuning *out);

/* Frees the plan (waits for the device).  NULL is accepted. */
int phprng_plan_destroy(phprng_plan *plan);

/* plan_create + plan_launch + plan_destroy for one batch. */
int phprng_generate_batch(phprng_ctx *ctx, const phprng_request *reqs, uint64_t nreq,
                          void *c_base, double *r_base, void *cuda_stream);

/* ---------------------------------------------------------------- serving */

/* A request loop over every stream of a context, kept in device memory
 * (continuous batching).  Requests arrive through phprng_server_submit, now
 * or at a stated future time on the phprng_clock_ns() clock (an open-loop
 * arrival schedule is replayed exactly).  A scheduler thread admits arrived
 * requests in FIFO order while their outputs fit in the output arena of
 * output_budget_bytes (the admission bound; a request then starts right
 * after the previous request of its stream), and whenever one of `inflight`
 * CUDA streams is free launches one batched persistent launch for everything
 * admitted since -- requests that arrive while others run join the next
 * launch and overlap them on the device.  Finished requests are handed back
 * by phprng_server_poll with their arrival and completion times; their
 * outputs stay in the arena until phprng_server_release.  While a server
 * runs, the context's other calls return PHPRNG_EINVAL. */
typedef struct phprng_server phprng_server;   /* opaque, library-owned */

typedef struct {
    uint64_t output_budget_bytes;  /* arena size: the admission bound on outstanding outputs */
    uint32_t max_batch;            /* requests per launch (0 = 4096) */
    uint32_t inflight;             /* launches in flight, one CUDA stream each (0 = 2, max 16) */
    uint32_t tile;                 /* numbers per tile; 0 = sized per launch: about one tile
                                      per resident warp, 256 to 4096 numbers (the lowest
                                      latency at light load) */
    uint32_t want_c;               /* nonzero: also store ciphertexts after each request's R */
} phprng_server_config;

typedef struct {
    uint64_t id, tag, inst;        /* request id (from submit), caller tag, stream */
    uint64_t start, len;           /* the request produced numbers start+1 .. start+len */
    const double *r;               /* device pointer to its R values (Eq. 9d) */
    const void *c;                 /* device pointer to its ciphertexts, or NULL */
    int64_t arrival_ns, done_ns;   /* arrival and completion on phprng_clock_ns() */
} phprng_completion;

typedef struct {
    uint64_t submitted, admitted, completed, batches, tiles, numbers;
    uint64_t max_waiting;          /* most requests seen waiting for admission at once */
    uint64_t waiting;              /* submitted and not yet admitted, now */
    uint64_t outstanding_bytes;    /* arena bytes held by admitted or unreleased requests */
} phprng_server_stats;

/* Monotonic clock of the server (CLOCK_MONOTONIC), nanoseconds. */
int64_t phprng_clock_ns(void);

/* Allocates the output arena (device), builds the skip table if needed and
 * starts the scheduler thread. */
int phprng_server_create(phprng_ctx *ctx, const phprng_server_config *cfg,
                         phprng_server **out);

/* Submits count requests (host arrays): stream inst[j], len[j] numbers
 * (1 <= len <= 2^32 and at most 65,536 tiles), optional tag[j] and optional
 * arrival_ns[j] (NULL:
 * now).  *first_id (nullable) receives the id of the first; ids are
 * consecutive.  PHPRNG_EBUDGET if one request alone exceeds the arena. */
int phprng_server_submit(phprng_server *srv, const uint64_t *inst, const uint64_t *len,
                         const uint64_t *tag, const int64_t *arrival_ns, uint64_t count,
                         uint64_t *first_id);

/* Moves up to max finished requests into out (waiting up to timeout_ns for
 * the first) and stores their number in *count. */
int phprng_server_poll(phprng_server *srv, phprng_completion *out, uint64_t max,
                       uint64_t *count, int64_t timeout_ns);

/* Copies finished request id's outputs (len doubles to r_dst, len
 * ciphertexts to c_dst; either NULL) into caller memory, host or device,
 * before it is released.  Synchronous. */
int phprng_server_copy(phprng_server *srv, uint64_t id, double *r_dst, void *c_dst);

/* Returns the output memory of finished requests to the arena. */
int phprng_server_release(phprng_server *srv, const uint64_t *ids, uint64_t count);

/* Counters of the server so far. */
int phprng_server_stats_get(phprng_server *srv, phprng_server_stats *out);

/* Stops the server: requests not yet admitted are dropped, admitted ones
 * finish; the streams' stored states are advanced to their served positions
 * (Eq. 7); the arena is freed.  NULL is accepted. */
int phprng_server_destroy(phprng_server *srv);

/* Sets instance inst's state: its next number is made from message m and skip
 * s by Eq. 9 as number pos+1 of its stream, and c is kept as the last
 * ciphertext.  The stream is redefined as the one through (m, s) at position
 * pos: its seed becomes the state pos steps earlier (Eq. 7 backwards: the
 * cycle position of s is a discrete logarithm on the host, the sum of the
 * skips in between comes from the prefix table; for the constant skip the
 * seed is m - pos s mod n with s0 = s), so phprng_seek,
 * phprng_skip, batched requests with offsets and the server all follow the
 * new stream.  With phprng_get_state this checkpoints and restores streams,
 * also into another context made from the same instance table (the seed then
 * comes out unchanged).  Limits: m < n, c < n, 1 <= s <= p-1.  Builds the
 * prefix table on first use; waits for work queued on cuda_stream and
 * returns with the state written. */
int phprng_set_state(phprng_ctx *ctx, uint64_t inst, uint64_t m, uint64_t s, uint64_t c, uint64_t pos,
                     void *cuda_stream);

/* Copies instance inst's parameters and current state to the host: the
 * returned phprng_instance holds {n, e, p, a, m, s} with m, s the current
 * message and skip; *pos_out (nullable) its stream position and *c_out
 * (nullable) the last ciphertext (0 before the first number).  Waits for
 * work queued on cuda_stream. */
int phprng_get_state(phprng_ctx *ctx, uint64_t inst, phprng_instance *state_out,
                     uint64_t *pos_out, uint64_t *c_out, void *cuda_stream);

/* ---------------------------------------------------------------- measurement */

/* Measures the current device's throughput for one instruction form and
 * stores operations per second in *ops_per_s (eight independent chains per
 * thread over a full-occupancy grid, timed with CUDA events on cuda_stream;
 * the call synchronizes).  which: 0 mul.lo.u32, 1 mad.hi.u32, 2 mad.wide.u32
 * (each 32-bit product half is the unit of the generator's roofline: forms
 * 0 and 1 make one half, form 2 two), 3 the generator's Montgomery product
 * mod a 32-bit prime, 4 fma.rn.f64, 5 the generator's window exponent
 * programs alone on 65,536 seeded 32-bit instances (Montgomery products per
 * second; draws the instances on the host first), 6 div.rn.f64 (FP64
 * division), 7 the generator's correctly rounded R = (c+1)/(n+1) built from
 * integers (Eq. 9d; numbers per second), 8 mul.wide.u32 (both halves), 9 the
 * Montgomery product with mul.lo and mul.hi in place of mul.wide, 10 the
 * Montgomery product by a constant (three multiplies), 11 a product by a
 * constant mod 2^31 - 1 with a precomputed quotient factor (Shoup's
 * method).  Allocates and frees small
 * device buffers.  The paper has no counterpart: this is the measurement used to
 * state the multiply-bound roofline of Eq. 9c. */
int phprng_microbench(int which, double *ops_per_s, void *cuda_stream);

/* ---------------------------------------------------------------- host only
 * These run on the CPU and need no GPU. */

/* 1 if n is prime, else 0: trial division by the primes below 256, then
 * the deterministic Rabin-Miller test with the paper's bases (2,3,5,7,11
 * below 2^32, the twelve primes up to 37 below 2^64), Implementation
 * section. */
int phprng_is_prime(uint64_t n);

/* Validates instances exactly as phprng_create does, without a GPU.
 * *bad_index (nullable) receives the first failing instance. */
int phprng_validate(int width, const phprng_instance *inst, uint64_t count, uint32_t flags,
                    uint64_t *bad_index);

/* Draws `count` instances from `seed` (Implementation section, seeding
 * paragraph, with a fixed seed in place of the system time): distinct
 * primes n in [2^31, 2^32) (width 32) or [2^63, 2^64) (width 64), safe
 * primes when PHPRNG_REQUIRE_SAFE_PRIME; e uniform in [3, n-2] with
 * gcd(e, n-1) = 1; m0 uniform in [0, n); s0 = a^L mod p with L uniform in
 * [0, p-2] (the stream skipped forward L steps from s = 1 by Eq. 7);
 * (p, a) = (2^31-1, 784588716).  Random source: SplitMix64.
 * out must hold count entries. */
int phprng_draw_instances(int width, uint64_t count, uint64_t seed, uint32_t flags,
                          phprng_instance *out);

#ifdef __cplusplus
}
#endif

#endif /* PHPRNG_H */
