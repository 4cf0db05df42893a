/*
 * phprng_oracle.c -- plain CPU oracle for the Pohlig-Hellman exponentiation-
 * cipher pseudorandom generator (P. D. Beale, "A new class of scalable
 * parallel pseudorandom number generators based on Pohlig-Hellman
 * exponentiation ciphers", arXiv:1411.2484).
 *
 * TEST INFRASTRUCTURE.  This is the slow, obviously-correct reference that the
 * CUDA library is checked against.  Only tests/, __graft_entry__.smoke() and
 * the CPU-baseline / reference leg of bench.py load it.  It shares no code,
 * header, table or constant with the CUDA library: every modular product is
 * the remainder of an exact integer product (the paper's definition of
 * "x = y mod z", Introduction), exponentiation is textbook repeated squaring,
 * and R is the C expression (double)(c+1) / (double)(n+1).
 *
 * Parity status of each function is stated in its comment ("pinned by ...").
 * The pins live in tests/test_oracle_pins.py and tests/golden/.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

/* x*y mod n, 0 <= result < n (Introduction: "x = y mod z means x is the
 * remainder of y upon division by z").  For n < 2^32 this is the paper's
 * one 64-bit multiply and one 64-bit mod (Implementation section, first
 * paragraph); for larger n the product is formed on 128 bits (the 64-bit
 * variant, Implementation section, last paragraph).
 * Pinned by: Python pow / exact integers in test_oracle_pins.py. */
uint64_t or_mulmod(uint64_t x, uint64_t y, uint64_t n)
{
    if (n <= 0xFFFFFFFFull && x < n && y < n)
        return (x * y) % n;
    return (uint64_t)(((u128)x * (u128)y) % (u128)n);
}

/* b^e mod n by repeated squaring, right-to-left over the bits of e
 * (Introduction: "method of repeated squaring").  Returns 1 mod n for e = 0.
 * Pinned by: Python pow, Fermat's little theorem, the decryption identity
 * Eq. 2, the Fig. 2 and Fig. 3 values. */
uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t n)
{
    uint64_t result = 1 % n;
    uint64_t base = b % n;
    while (e) {
        if (e & 1) result = or_mulmod(result, base, n);
        base = or_mulmod(base, base, n);
        e >>= 1;
    }
    return result;
}

/* Eq. 9d: R = (c+1)/(n+1) as one floating-point division in double.
 * For n < 2^32 both operands are exact doubles and R is the correctly
 * rounded quotient.  For 64-bit n each operand is first rounded to double
 * (the C conversion), then divided: the reading of Eq. 9d for 64-bit moduli.
 * Pinned by: Python Fraction / float division in test_oracle_pins.py. */
double or_real(uint64_t c, uint64_t n)
{
    return (double)(c + 1) / (double)(n + 1);
}

/* Eq. 9a-9e applied `count` times to the state st[0] = m, st[1] = s:
 *   s := a s mod p;  m := (m + s) mod n;  c := m^e mod n;  R := (c+1)/(n+1).
 * The k-th output (k = 0..count-1) goes to c_out[k], r_out[k] (either may be
 * NULL).  On return st holds the state after the last output.
 * Pinned by: the hand-worked n=23 table (tests/golden/tiny_n23_eq9.txt), the
 * period n(p-1) and the exact (p-1)-fold multiplicity of every ciphertext on
 * tiny instances (Section "Message skipping algorithms"), Fig. 2 values. */
void or_generate(uint64_t n, uint64_t e, uint64_t p, uint64_t a,
                 uint64_t *st, uint64_t count, uint64_t *c_out, double *r_out)
{
    uint64_t m = st[0], s = st[1];
    for (uint64_t k = 0; k < count; ++k) {
        s = or_mulmod(a, s, p);                      /* Eq. 9a */
        m = (uint64_t)(((u128)m + s) % n);           /* Eq. 9b */
        uint64_t c = or_powmod(m, e, n);             /* Eq. 9c */
        if (c_out) c_out[k] = c;
        if (r_out) r_out[k] = or_real(c, n);         /* Eq. 9d */
    }
    st[0] = m;
    st[1] = s;
}

/* Eq. 7 with the current state (m, s) taken as the origin: advance k steps.
 * q = floor(k/(p-1)), r = k mod (p-1);
 *   s' = s a^r mod p;
 *   m' = (m + q p(p-1)/2 + sum_{j=1..r} (s a^j mod p)) mod n.
 * The sum is formed by stepping the skip generator r times.
 * Pinned by: direct stepping with or_generate on tiny and 32-bit instances. */
void or_skip_stepping(uint64_t n, uint64_t p, uint64_t a, uint64_t *st, uint64_t k)
{
    uint64_t q = k / (p - 1), r = k % (p - 1);
    uint64_t m = st[0], s = st[1];
    u128 half_cycle = ((u128)p * (u128)(p - 1)) / 2;          /* p(p-1)/2 */
    uint64_t b = (uint64_t)(half_cycle % n);
    uint64_t add = (uint64_t)(((u128)(q % n) * b) % n);
    uint64_t x = s;
    u128 sum = 0;
    for (uint64_t j = 1; j <= r; ++j) {
        x = or_mulmod(a, x, p);
        sum += x;
    }
    st[0] = (uint64_t)(((u128)m + add + sum % n) % n);
    st[1] = or_mulmod(s, or_powmod(a, r, p), p);            /* Eq. 7a */
}

/* Coarse prefix table of the skip generator's cycle:
 *   table[j] = sum_{i=1..j*stride} (a^i mod p),  j = 0 .. (p-1)/stride.
 * Built by one plain loop over the cycle (Eq. 6b with s0 = 1).  nent must be
 * (p-1)/stride + 1.  The last cycle sum is p(p-1)/2 (proof of the period,
 * "Message skipping algorithms").
 * Pinned by: table[(p-1)/stride] = p(p-1)/2 when stride divides p-1, and
 * brute-force sums on tiny p. */
void or_prefix_table(uint64_t p, uint64_t a, uint64_t stride, uint64_t *table, uint64_t nent)
{
    uint64_t x = 1, sum = 0;
    table[0] = 0;
    for (uint64_t i = 1, j = 1; j < nent; ++i) {
        x = or_mulmod(a, x, p);
        sum += x;
        if (i % stride == 0) table[j++] = sum;
    }
}

/* Pref(t) = sum_{i=1..t} (a^i mod p) for 0 <= t <= p-1, from the coarse
 * table plus at most stride-1 plain steps. */
uint64_t or_pref(uint64_t p, uint64_t a, const uint64_t *table, uint64_t stride, uint64_t t)
{
    uint64_t j = t / stride;
    uint64_t sum = table[j];
    uint64_t x = or_powmod(a, j * stride, p);
    for (uint64_t i = j * stride + 1; i <= t; ++i) {
        x = or_mulmod(a, x, p);
        sum += x;
    }
    return sum;
}

/* State after t steps from the seed (m0, s0 = a^L0 mod p), Eq. 7:
 * q = floor(t/(p-1)), r = t mod (p-1),
 *   s_t = s0 a^r mod p = a^(L0+r) mod p,
 *   m_t = (m0 + q p(p-1)/2 + sum_{j=1..r} a^(L0+j) mod p) mod n,
 * where the sum is Pref(L0+r) - Pref(L0), wrapping once around the cycle of
 * length p-1 (a^(p-1) = 1, Pref(p-1) = p(p-1)/2) when L0 + r > p-1.
 * Pinned by: or_skip_stepping and direct stepping. */
void or_state_at(uint64_t n, uint64_t p, uint64_t a, uint64_t m0, uint64_t L0,
                 uint64_t t, const uint64_t *table, uint64_t stride, uint64_t *st_out)
{
    uint64_t q = t / (p - 1), r = t % (p - 1);
    u128 half_cycle = ((u128)p * (u128)(p - 1)) / 2;
    uint64_t b = (uint64_t)(half_cycle % n);
    uint64_t add = (uint64_t)(((u128)(q % n) * b) % n);
    u128 sum;
    uint64_t hi = L0 + r;
    if (hi <= p - 1) {
        sum = (u128)or_pref(p, a, table, stride, hi) - or_pref(p, a, table, stride, L0);
    } else {
        sum = half_cycle - or_pref(p, a, table, stride, L0)
            + or_pref(p, a, table, stride, hi - (p - 1));
    }
    st_out[0] = (uint64_t)(((u128)m0 + add + sum % n) % n);
    st_out[1] = or_powmod(a, L0 + r, p);
}

/* Discrete logarithm base a modulo p by Shanks' baby-step giant-step:
 * finds L in [0, p-2] with a^L = s mod p for each query s (a must be a
 * primitive root, s in [1, p-1]).  L_out[i] = UINT64_MAX when not found.
 * Used only to place seeds s0 on the skip cycle for or_state_at.
 * Pinned by: pow(a, L, p) == s in the tests. */
int or_dlog_many(uint64_t p, uint64_t a, const uint64_t *s, uint64_t cnt, uint64_t *L_out)
{
    uint64_t order = p - 1;
    uint64_t M = 1;
    while (M * M < order) ++M;
    uint64_t cap = 1;
    while (cap < 2 * M) cap <<= 1;
    uint64_t *key = (uint64_t *)malloc(cap * sizeof(uint64_t));
    uint64_t *val = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!key || !val) { free(key); free(val); return -1; }
    for (uint64_t i = 0; i < cap; ++i) key[i] = 0;   /* 0 is never a power of a */
    uint64_t x = 1;
    for (uint64_t j = 0; j < M; ++j) {               /* baby steps a^j */
        uint64_t h = (x * 0x9E3779B97F4A7C15ull) & (cap - 1);
        while (key[h] != 0 && key[h] != x) h = (h + 1) & (cap - 1);
        if (key[h] == 0) { key[h] = x; val[h] = j; }
        x = or_mulmod(x, a, p);
    }
    /* giant step factor a^(-M) = a^(p-1-M mod p-1) */
    uint64_t g = or_powmod(a, (order - (M % order)) % order, p);
    for (uint64_t q = 0; q < cnt; ++q) {
        uint64_t y = s[q] % p;
        L_out[q] = UINT64_MAX;
        for (uint64_t i = 0; i <= M && y != 0; ++i) {
            uint64_t h = (y * 0x9E3779B97F4A7C15ull) & (cap - 1);
            while (key[h] != 0) {
                if (key[h] == y) { L_out[q] = (i * M + val[h]) % order; break; }
                h = (h + 1) & (cap - 1);
            }
            if (L_out[q] != UINT64_MAX) break;
            y = or_mulmod(y, g, p);
        }
    }
    free(key);
    free(val);
    return 0;
}

/* Exact u128 -> double, correctly rounded (the compiler's conversion). */
static double u128_to_double(u128 v) { return (double)v; }

/* Per-stream statistics of one call's ciphertexts (definitions of this
 * library's fused consumer mode; the paper's frequency test, Tests section,
 * motivates the histogram):
 *   X = sum (c+1),  Y = sum (c+1)^2        (exact 128-bit integers)
 *   hist[b] = #{k : floor(256 R_k) = b}, R_k from or_real (b = 255 for R = 1)
 *   mean = RN(RN(X) / RN(N (n+1)))
 *   var  = RN(RN(N Y - X^2) / RN(N (N-1) (n+1)^2))   (0 when N < 2)
 * xy_out = {X lo, X hi, Y lo, Y hi}; mv_out = {mean, var}.
 * Pinned by: full-period closed forms on tiny instances (every c appears p-1
 * times, so X = (p-1) n(n+1)/2 and Y = (p-1) n(n+1)(2n+1)/6). */
void or_stats(const uint64_t *c, uint64_t N, uint64_t n,
              uint64_t *xy_out, uint32_t *hist, double *mv_out)
{
    u128 X = 0, Y = 0;
    for (int b = 0; b < 256; ++b) hist[b] = 0;
    for (uint64_t k = 0; k < N; ++k) {
        u128 v = (u128)c[k] + 1;
        X += v;
        Y += v * v;
        double R = or_real(c[k], n);
        int b = (int)(R * 256.0);
        if (b > 255) b = 255;
        hist[b] += 1;
    }
    xy_out[0] = (uint64_t)X; xy_out[1] = (uint64_t)(X >> 64);
    xy_out[2] = (uint64_t)Y; xy_out[3] = (uint64_t)(Y >> 64);
    u128 n1 = (u128)n + 1;
    mv_out[0] = N ? u128_to_double(X) / u128_to_double((u128)N * n1) : 0.0;
    if (N >= 2) {
        u128 num = (u128)N * Y - X * X;
        u128 den = (u128)N * (N - 1) * n1 * n1;
        mv_out[1] = u128_to_double(num) / u128_to_double(den);
    } else {
        mv_out[1] = 0.0;
    }
}

/* Adjacent-stream product sum for the interstream ordering of the paper's
 * correlation tests ("Message skipping algorithms", last item):
 *   Z = sum_k (ca_k + 1)(cb_k + 1),  corr = RN(RN(Z) / RN(N (na+1)(nb+1))).
 * z_out = {Z lo, Z hi}.
 * Pinned by: identical streams give Z = Y; Cauchy-Schwarz Z^2 <= Ya Yb. */
void or_corr(const uint64_t *ca, const uint64_t *cb, uint64_t N,
             uint64_t na, uint64_t nb, uint64_t *z_out, double *corr_out)
{
    u128 Z = 0;
    for (uint64_t k = 0; k < N; ++k)
        Z += ((u128)ca[k] + 1) * ((u128)cb[k] + 1);
    z_out[0] = (uint64_t)Z; z_out[1] = (uint64_t)(Z >> 64);
    *corr_out = N ? u128_to_double(Z) /
                    u128_to_double((u128)N * ((u128)na + 1) * ((u128)nb + 1)) : 0.0;
}

/* Serial-test histogram (Tests section, items 1-5: the one-dimensional
 * frequency test and the two- to five-dimensional serial tests).  One
 * stream's numbers R_k = or_real(c_k) in order, grouped into consecutive
 * non-overlapping D-tuples (R_{tD+1}, ..., R_{tD+D}) for t = 0 ..
 * floor(N/D)-1 (a shorter remainder is left out); each coordinate falls in bin
 * floor(B R) of B bins per dimension (B - 1 for R = 1), and the tuple adds one
 * to hist[b_0 + B b_1 + ... + B^(D-1) b_(D-1)] (hist has B^D entries and is
 * added to, not cleared).
 * Pinned by: the full-period one-dimensional histogram of tiny instances
 * (every c appears p-1 times, bins counted with exact rationals); the tuple
 * count floor(N/D); the marginal of a coordinate equal to the one-dimensional
 * histogram of every D-th number; bins of exact multiples of 1/B. */
void or_serial_hist(const uint64_t *c, uint64_t N, uint64_t n, int D, uint64_t B,
                    uint64_t *hist)
{
    for (uint64_t t = 0; t < N / (uint64_t)D; ++t) {
        uint64_t idx = 0, scale = 1;
        for (int d = 0; d < D; ++d) {
            double R = or_real(c[t * (uint64_t)D + (uint64_t)d], n);
            uint64_t b = (uint64_t)(R * (double)B);
            if (b >= B) b = B - 1;
            idx += b * scale;
            scale *= B;
        }
        hist[idx] += 1;
    }
}

/* Interstream serial test (Tests section, interstream correlations): the
 * numbers of Np streams are taken in the paper's interleaved order -- the
 * first number of every stream, stream 0 to Np-1, then the second of every
 * stream, and so on -- and that one sequence S[j Np + a] = R_(j+1) of stream a
 * is cut into consecutive non-overlapping D-tuples (a remainder of fewer
 * than D is left out), each adding one to hist[b_1 + B b_2 + ...] with
 * b = floor(B R).  c holds the streams' ciphertexts instance-major (stream a,
 * number j at c[a L + j]) and nmod[a] the moduli.
 * Pinned by: Np = 1 equals or_serial_hist; the sequence built by hand in
 * Python on small cases; for D = 1 the sum of the streams' own histograms. */
void or_interstream_serial_hist(const uint64_t *c, const uint64_t *nmod, uint64_t Np, uint64_t L, int D,
                                uint64_t B, uint64_t *hist)
{
    uint64_t total = Np * L;
    for (uint64_t t = 0; t < total / (uint64_t)D; ++t) {
        uint64_t idx = 0, scale = 1;
        for (int d = 0; d < D; ++d) {
            uint64_t q = t * (uint64_t)D + (uint64_t)d;    /* position in the interleaved sequence */
            uint64_t a = q % Np, j = q / Np;
            double R = or_real(c[a * L + j], nmod[a]);
            uint64_t b = (uint64_t)(R * (double)B);
            if (b >= B) b = B - 1;
            idx += b * scale;
            scale *= B;
        }
        hist[idx] += 1;
    }
}

/* Poker test (Tests section: five cards, ten denominations).  One stream's
 * numbers in consecutive non-overlapping 5-tuples (a remainder of fewer than
 * five is left out); card k of a hand has denomination floor(10 R_k); the
 * hand adds one to hist[category] with categories 0 all different, 1 one
 * pair, 2 two pairs, 3 three of a kind, 4 full house, 5 four of a kind,
 * 6 five of a kind (hist has 7 entries and is added to).
 * Pinned by: hands built from chosen denominations; the hand count floor(N/5);
 * the category frequencies of a long stream against the exact probabilities
 * (0.3024, 0.504, 0.108, 0.072, 0.009, 0.0045, 0.0001). */
void or_poker_hist(const uint64_t *c, uint64_t N, uint64_t n, uint64_t *hist)
{
    for (uint64_t t = 0; t < N / 5; ++t) {
        int count[10] = {0};
        for (int k = 0; k < 5; ++k) {
            int d = (int)(or_real(c[t * 5 + (uint64_t)k], n) * 10.0);
            if (d > 9) d = 9;
            count[d] += 1;
        }
        int pairs = 0, threes = 0, fours = 0, fives = 0;
        for (int d = 0; d < 10; ++d) {
            if (count[d] == 2) ++pairs;
            if (count[d] == 3) ++threes;
            if (count[d] == 4) ++fours;
            if (count[d] == 5) ++fives;
        }
        int cat;
        if (fives) cat = 6;
        else if (fours) cat = 5;
        else if (threes && pairs) cat = 4;
        else if (threes) cat = 3;
        else if (pairs == 2) cat = 2;
        else if (pairs == 1) cat = 1;
        else cat = 0;
        hist[cat] += 1;
    }
}

/* Runs test (Tests section: runs of 0's, R <= 0.5, and 1's, R > 0.5).  One
 * stream's numbers in order give bits b_k = (R_k > 0.5); every maximal run of
 * equal bits that ends before the last number adds one to
 * hist[b * Lmax + min(L, Lmax) - 1] (L its length; the run still open at the
 * last number is left out, the first run starts at the first number).  hist
 * has 2 Lmax entries and is added to.
 * Pinned by: bit patterns built from chosen c; total length of the counted
 * runs = N minus the open run; run-length frequencies of a long stream
 * against the probabilities 2^-L of fair independent bits. */
void or_runs_hist(const uint64_t *c, uint64_t N, uint64_t n, int Lmax, uint64_t *hist)
{
    if (N == 0) return;
    int bit = or_real(c[0], n) > 0.5;
    uint64_t len = 1;
    for (uint64_t k = 1; k < N; ++k) {
        int b = or_real(c[k], n) > 0.5;
        if (b == bit) {
            ++len;
            continue;
        }
        hist[(uint64_t)bit * (uint64_t)Lmax + (len < (uint64_t)Lmax ? len : (uint64_t)Lmax) - 1] += 1;
        bit = b;
        len = 1;
    }
}

/* Full-period D-dimensional pattern by enumeration (the O(p L0) method that
 * follows Eq. 7): over the full period n(p-1), ciphertext c_k = c0 occurs
 * p-1 times, once with each skip s_(k+1) = s in (Z/pZ)*, with message
 * m = c0^d mod n (d = e^-1 mod n-1, Eq. 2); the succeeding points are
 * c_(k+j) = (m + s + a s + ... + a^(j-1) s (each term mod p))^e mod n.  For every
 * c0 in [c_lo, c_lo + L0) and every s in 1 .. p-1 the point (c_(k+1), ...,
 * c_(k+D-1)) adds one to hist[b_1 + nb b_2 + ... + nb^(D-2) b_(D-1)] with
 * b_j = floor(c_(k+j) / L1), L1 = ceil(n / nb) (hist has nb^(D-1) entries and is
 * added to).
 * Pinned by: the same histogram counted by brute force over a whole period
 * of tiny instances (or_generate, every k with c_k in the range); for D = 2
 * and the whole range of c0, each bin holds p-1 times its count of values. */
void or_pattern_hist(uint64_t n, uint64_t e, uint64_t p, uint64_t a, uint64_t c_lo,
                     uint64_t L0, int D, uint64_t nb, uint64_t *hist)
{
    /* d = e^-1 mod (n-1) by the extended Euclidean algorithm */
    int64_t r0 = (int64_t)(n - 1), r1 = (int64_t)(e % (n - 1)), t0 = 0, t1 = 1;
    while (r1) {
        int64_t q = r0 / r1, tmp;
        tmp = r0 - q * r1; r0 = r1; r1 = tmp;
        tmp = t0 - q * t1; t0 = t1; t1 = tmp;
    }
    uint64_t d = (uint64_t)(t0 < 0 ? t0 + (int64_t)(n - 1) : t0);
    uint64_t L1 = (n + nb - 1) / nb;
    for (uint64_t c0 = c_lo; c0 < c_lo + L0; ++c0) {
        uint64_t m = or_powmod(c0, d, n);
        for (uint64_t s = 1; s < p; ++s) {
            uint64_t acc = m, t = s, idx = 0, scale = 1;
            for (int j = 1; j < D; ++j) {
                acc = (uint64_t)(((u128)acc + t) % n);
                uint64_t c = or_powmod(acc, e, n);
                idx += (c / L1) * scale;
                scale *= nb;
                t = or_mulmod(a, t, p);
            }
            hist[idx] += 1;
        }
    }
}

/* Full-period pattern of the constant-skip generator ("Message skipping
 * algorithms": s_k = b, so m_k = m_0 + k b mod n, period n; b = 1 is the unit
 * skip, a block cipher in counter mode): every c0 occurs once per period, with
 * message m = c0^d mod n, and the tuple that starts at c0 continues with
 * c_(k+j) = (m + j b)^e mod n.  For every c0 in [c_lo, c_lo + L0) the point
 * (c_(k+1), ..., c_(k+D-1)) adds one to hist[b_1 + nb b_2 + ...] with
 * b_j = floor(c_(k+j) / L1), L1 = ceil(n / nb) (hist added to).
 * Pinned by: brute-force counts over a whole period of m_k = m_0 + k b. */
void or_pattern_const_hist(uint64_t n, uint64_t e, uint64_t b, uint64_t c_lo, uint64_t L0, int D,
                           uint64_t nb, uint64_t *hist)
{
    int64_t r0 = (int64_t)(n - 1), r1 = (int64_t)(e % (n - 1)), t0 = 0, t1 = 1;
    while (r1) {
        int64_t q = r0 / r1, tmp;
        tmp = r0 - q * r1; r0 = r1; r1 = tmp;
        tmp = t0 - q * t1; t0 = t1; t1 = tmp;
    }
    uint64_t d = (uint64_t)(t0 < 0 ? t0 + (int64_t)(n - 1) : t0);
    uint64_t L1 = (n + nb - 1) / nb;
    for (uint64_t c0 = c_lo; c0 < c_lo + L0; ++c0) {
        uint64_t m = or_powmod(c0, d, n), idx = 0, scale = 1;
        for (int j = 1; j < D; ++j) {
            uint64_t mj = (uint64_t)(((u128)m + (u128)j * (b % n)) % n);
            idx += (or_powmod(mj, e, n) / L1) * scale;
            scale *= nb;
        }
        hist[idx] += 1;
    }
}

/* Full-period patterns over a region near the origin (the paper's Figs. 2-4:
 * magnified squares and slabs): as or_pattern_hist and or_pattern_const_hist,
 * but with the cell width L1 given and only the tuples whose successors all
 * lie below nb L1 counted (the others are left out), so that hist[b_1 + nb b_2
 * + ...], b_j = floor(c_(k+j) / L1), covers the region [0, nb L1)^(D-1) of the
 * successors for the starting values c0 in [c_lo, c_lo + L0).  With
 * L1 = ceil(n / nb) nothing is left out and the results equal the full-range
 * functions.  b = 0 in or_pattern_region_hist selects the pseudorandom skip
 * (p, a); or_pattern_const_region_hist takes the constant skip b.
 * Pinned by: the full-range reduction; brute-force counts over whole periods
 * of tiny instances; the paper's Fig. 2 crib pairs for the unit skip; the
 * Fig. 3 properties (each pair at most once, none on the diagonal). */
static uint64_t or_inverse_exponent(uint64_t n, uint64_t e)
{
    int64_t r0 = (int64_t)(n - 1), r1 = (int64_t)(e % (n - 1)), t0 = 0, t1 = 1;
    while (r1) {
        int64_t q = r0 / r1, tmp;
        tmp = r0 - q * r1; r0 = r1; r1 = tmp;
        tmp = t0 - q * t1; t0 = t1; t1 = tmp;
    }
    return (uint64_t)(t0 < 0 ? t0 + (int64_t)(n - 1) : t0);
}

void or_pattern_region_hist(uint64_t n, uint64_t e, uint64_t p, uint64_t a, uint64_t c_lo,
                            uint64_t L0, int D, uint64_t nb, uint64_t L1, uint64_t *hist)
{
    uint64_t d = or_inverse_exponent(n, e);
    for (uint64_t c0 = c_lo; c0 < c_lo + L0; ++c0) {
        uint64_t m = or_powmod(c0, d, n);
        for (uint64_t s = 1; s < p; ++s) {
            uint64_t acc = m, t = s, idx = 0, scale = 1;
            int inside = 1;
            for (int j = 1; j < D; ++j) {
                acc = (uint64_t)(((u128)acc + t) % n);
                uint64_t c = or_powmod(acc, e, n);
                if (c / L1 >= nb) inside = 0;
                idx += (c / L1) * scale;
                scale *= nb;
                t = or_mulmod(a, t, p);
            }
            if (inside) hist[idx] += 1;
        }
    }
}

void or_pattern_const_region_hist(uint64_t n, uint64_t e, uint64_t b, uint64_t c_lo, uint64_t L0, int D,
                                  uint64_t nb, uint64_t L1, uint64_t *hist)
{
    uint64_t d = or_inverse_exponent(n, e);
    for (uint64_t c0 = c_lo; c0 < c_lo + L0; ++c0) {
        uint64_t m = or_powmod(c0, d, n), idx = 0, scale = 1;
        int inside = 1;
        for (int j = 1; j < D; ++j) {
            uint64_t mj = (uint64_t)(((u128)m + (u128)j * (b % n)) % n);
            uint64_t c = or_powmod(mj, e, n);
            if (c / L1 >= nb) inside = 0;
            idx += (c / L1) * scale;
            scale *= nb;
        }
        if (inside) hist[idx] += 1;
    }
}

/* Collision test (Tests section: 2^14 numbers into 2^20 bins).  One stream's
 * numbers in consecutive non-overlapping segments of S (a remainder of fewer
 * than S is left out); number k falls in bin floor(B R_k); a number is a
 * collision when its bin already holds an earlier number of the segment;
 * the segment's collision count C adds one to hist[min(C, H-1)] (hist has H
 * entries and is added to).
 * Pinned by: segments built from chosen bins; the mean collision count of a
 * long stream against its exact expectation S - B (1 - (1 - 1/B)^S). */
void or_collision_hist(const uint64_t *c, uint64_t N, uint64_t n, uint64_t S, uint64_t B,
                       uint64_t H, uint64_t *hist)
{
    unsigned char *seen = (unsigned char *)calloc(B, 1);
    if (!seen) return;
    for (uint64_t g = 0; g + S <= N; g += S) {
        uint64_t C = 0;
        for (uint64_t k = g; k < g + S; ++k) {
            uint64_t b = (uint64_t)(or_real(c[k], n) * (double)B);
            if (b >= B) b = B - 1;
            if (seen[b]) ++C;
            seen[b] = 1;
        }
        hist[C < H ? C : H - 1] += 1;
        for (uint64_t k = g; k < g + S; ++k) {
            uint64_t b = (uint64_t)(or_real(c[k], n) * (double)B);
            if (b >= B) b = B - 1;
            seen[b] = 0;
        }
    }
    free(seen);
}

/* ---- threaded harness: many independent instances (parameter splitting,
 * Introduction: each process owns its own prime modulus) ------------------ */
typedef struct {
    const uint64_t *params;   /* [count][6] = n, e, p, a, m, s */
    uint64_t lo, hi, per_inst;
    uint64_t *c_out;          /* [count][per_inst] or NULL */
    double *r_out;            /* [count][per_inst] or NULL */
    uint64_t *state_out;      /* [count][2] or NULL */
    uint64_t sink;
} or_job;

static void *or_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    uint64_t sink = 0;
    uint64_t *cbuf = NULL;
    if (!j->c_out) cbuf = (uint64_t *)malloc(j->per_inst * sizeof(uint64_t));
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        const uint64_t *P = j->params + 6 * i;
        uint64_t st[2] = {P[4], P[5]};
        uint64_t *c = j->c_out ? j->c_out + i * j->per_inst : cbuf;
        double *r = j->r_out ? j->r_out + i * j->per_inst : NULL;
        or_generate(P[0], P[1], P[2], P[3], st, j->per_inst, c, r);
        if (!j->c_out && c) for (uint64_t k = 0; k < j->per_inst; ++k) sink ^= c[k];
        if (j->state_out) { j->state_out[2 * i] = st[0]; j->state_out[2 * i + 1] = st[1]; }
    }
    free(cbuf);
    j->sink = sink;
    return NULL;
}

/* Runs or_generate for `count` instances over `threads` POSIX threads
 * (instances split into contiguous ranges).  Returns an XOR of the
 * ciphertexts when c_out is NULL (so the work cannot be discarded). */
uint64_t or_generate_many(const uint64_t *params, uint64_t count, uint64_t per_inst,
                          int threads, uint64_t *c_out, double *r_out, uint64_t *state_out)
{
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > count) threads = count ? (int)count : 1;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    or_job *jobs = (or_job *)malloc(sizeof(or_job) * threads);
    uint64_t sink = 0;
    for (int t = 0; t < threads; ++t) {
        jobs[t].params = params;
        jobs[t].lo = count * t / threads;
        jobs[t].hi = count * (t + 1) / threads;
        jobs[t].per_inst = per_inst;
        jobs[t].c_out = c_out; jobs[t].r_out = r_out; jobs[t].state_out = state_out;
        jobs[t].sink = 0;
        pthread_create(&tid[t], NULL, or_worker, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) { pthread_join(tid[t], NULL); sink ^= jobs[t].sink; }
    free(tid);
    free(jobs);
    return sink;
}
