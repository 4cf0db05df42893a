// hostnt.cpp -- host instance layer: primality, validation, seeding and the
// per-instance constants the kernels read.
//
// Beale, arXiv:1411.2484, Implementation section: every process gets its own
// prime modulus n (Rabin-Miller, deterministic with the bases 2,3,5,7,11 below
// 2^32 and the twelve primes up to 37 below 2^64, after trial division by
// small primes), an exponent e coprime to n-1 (Eq. 1, Eq. 2), and a skip
// generator (p, a) with p < n prime and a a primitive root mod p (Eq. 5).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "arith.cuh"
#include "internal.h"

namespace phprng {

typedef unsigned __int128 u128;

uint64_t mulmod(uint64_t x, uint64_t y, uint64_t n)
{
    return (uint64_t)((u128)x * y % n);
}

uint64_t powmod(uint64_t b, uint64_t e, uint64_t n)
{
    uint64_t r = 1 % n;
    b %= n;
    while (e) {
        if (e & 1) r = mulmod(r, b, n);
        b = mulmod(b, b, n);
        e >>= 1;
    }
    return r;
}

uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) { uint64_t t = a % b; a = b; b = t; }
    return a;
}

int bitlen(uint64_t x)
{
    return x ? 64 - __builtin_clzll(x) : 0;
}

// Newton iteration x <- x (2 - n x): each step doubles the number of correct
// low bits; x = n is right mod 8 for odd n, so five steps reach 64 bits.
uint64_t inv_mod_2_64(uint64_t n)
{
    uint64_t x = n;
    for (int i = 0; i < 5; ++i) x *= 2 - n * x;
    return x;
}

static const uint32_t kSmallPrimes[] = {
    2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71, 73, 79, 83, 89,
    97, 101, 103, 107, 109, 113, 127, 131, 137, 139, 149, 151, 157, 163, 167, 173, 179, 181,
    191, 193, 197, 199, 211, 223, 227, 229, 233, 239, 241, 251};

// Strong probable prime to base g (the Rabin-Miller condition of the
// Implementation section): with n - 1 = 2^r t, t odd, either g^t = 1 or
// g^(2^j t) = n-1 for some 0 <= j < r.
static bool strong_probable_prime(uint64_t n, uint64_t g)
{
    uint64_t t = n - 1;
    int r = 0;
    while ((t & 1) == 0) { t >>= 1; ++r; }
    uint64_t x = powmod(g, t, n);
    if (x == 1 || x == n - 1) return true;
    for (int j = 1; j < r; ++j) {
        x = mulmod(x, x, n);
        if (x == n - 1) return true;
    }
    return false;
}

bool is_prime(uint64_t n)
{
    if (n < 2) return false;
    for (uint32_t q : kSmallPrimes) {          // trial division first
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    if (n < 256ull * 256ull) return true;      // no factor below 256 and n < 256^2
    static const uint64_t b32[] = {2, 3, 5, 7, 11};
    static const uint64_t b64[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < (1ull << 32)) {
        for (uint64_t g : b32) if (!strong_probable_prime(n, g)) return false;
    } else {
        for (uint64_t g : b64) if (!strong_probable_prime(n, g)) return false;
    }
    return true;
}

// A nontrivial factor of the odd composite x: Pollard's rho with Brent's
// cycle detection (R. P. Brent, "An improved Monte Carlo factorization
// algorithm", BIT 20, 1980), iterating y -> y^2 + c mod x and taking gcds of
// products of |x_i - y| over batches of 128 steps; a new c when a batch
// collapses to x.
static uint64_t rho_factor(uint64_t x)
{
    for (uint64_t c = 1;; ++c) {
        uint64_t y = 2, g = 1, q = 1, ys = 2, xs = 2;
        for (uint64_t r = 1; g == 1; r <<= 1) {
            xs = y;
            for (uint64_t i = 0; i < r; ++i) y = (mulmod(y, y, x) + c) % x;
            for (uint64_t k = 0; k < r && g == 1; k += 128) {
                ys = y;
                for (uint64_t i = 0; i < 128 && i < r - k; ++i) {
                    y = (mulmod(y, y, x) + c) % x;
                    q = mulmod(q, xs > y ? xs - y : y - xs, x);
                }
                g = gcd64(q, x);
            }
        }
        if (g == x) {                              // the batch overshot: step singly
            do {
                ys = (mulmod(ys, ys, x) + c) % x;
                g = gcd64(xs > ys ? xs - ys : ys - xs, x);
            } while (g == 1);
        }
        if (g != x) return g;
    }
}

static void factor_into(uint64_t x, std::vector<uint64_t> &f)
{
    if (x == 1) return;
    if (is_prime(x)) {
        f.push_back(x);
        return;
    }
    const uint64_t d = rho_factor(x);
    factor_into(d, f);
    factor_into(x / d, f);
}

// The distinct prime factors of x, ascending: trial division by the primes
// below 2^16 (by odd numbers), then Pollard's rho on what remains, so that
// p - 1 of a 63-bit skip prime factors in well under a second.
std::vector<uint64_t> prime_factors(uint64_t x)
{
    std::vector<uint64_t> f;
    for (uint64_t d = 2; d < 65536 && d * d <= x; d += (d == 2 ? 1 : 2)) {
        if (x % d == 0) {
            f.push_back(d);
            while (x % d == 0) x /= d;
        }
    }
    if (x > 1) {
        std::vector<uint64_t> big;
        factor_into(x, big);
        f.insert(f.end(), big.begin(), big.end());
    }
    std::sort(f.begin(), f.end());
    f.erase(std::unique(f.begin(), f.end()), f.end());
    return f;
}

// a is a primitive root mod prime p iff a^((p-1)/q) != 1 for every prime q | p-1.
bool is_primitive_root(uint64_t a, uint64_t p)
{
    if (a % p == 0) return false;
    for (uint64_t q : prime_factors(p - 1))
        if (powmod(a, (p - 1) / q, p) == 1) return false;
    return true;
}

// Discrete logarithms base a modulo p (a a primitive root): the
// Pohlig-Hellman reduction to the prime-order subgroups of (Z/pZ)*, digit by
// digit, with Shanks' baby-step giant-step in each subgroup, then the Chinese
// remainder theorem.  The baby-step tables depend only on (p, a), so one
// solver serves every seed of a context.  Used to place seeds s0 on the skip
// cycle so that Eq. 7 can be evaluated from the prefix table.
struct DlogSolver {
    struct Factor {
        uint64_t q, qk;
        int k;
        uint64_t gq, m, gm_inv;
        std::unordered_map<uint64_t, uint64_t> baby;
    };
    uint64_t p, a, N;
    std::vector<Factor> f;

    DlogSolver(uint64_t p_, uint64_t a_) : p(p_), a(a_), N(p_ - 1)
    {
        uint64_t rest = N;
        for (uint64_t q : prime_factors(N)) {
            Factor F;
            F.q = q; F.k = 0; F.qk = 1;
            while (rest % q == 0) { rest /= q; F.qk *= q; ++F.k; }
            F.gq = powmod(a, N / q, p);                   // generator of the order-q subgroup
            F.m = 1;
            while (F.m * F.m < q) ++F.m;
            F.baby.reserve(F.m * 2);
            uint64_t v = 1;
            for (uint64_t j = 0; j < F.m; ++j) {
                F.baby.emplace(v, j);
                v = mulmod(v, F.gq, p);
            }
            F.gm_inv = powmod(powmod(F.gq, F.m, p), p - 2, p);
            f.push_back(std::move(F));
        }
    }

    bool solve(uint64_t s, uint64_t *L) const
    {
        s %= p;
        if (s == 0) return false;
        uint64_t x = 0, mod = 1;
        for (const Factor &F : f) {
            uint64_t xq = 0, qj = 1;
            for (int j = 0; j < F.k; ++j) {
                // h = (s a^-xq)^(N / q^(j+1)) lies in the order-q subgroup
                uint64_t a_inv_xq = powmod(powmod(a, xq, p), p - 2, p);
                uint64_t h = powmod(mulmod(s, a_inv_xq, p), N / (qj * F.q), p);
                uint64_t y = h, d = UINT64_MAX;
                for (uint64_t i = 0; i <= F.m; ++i) {
                    auto it = F.baby.find(y);
                    if (it != F.baby.end()) { d = (i * F.m + it->second) % F.q; break; }
                    y = mulmod(y, F.gm_inv, p);
                }
                if (d == UINT64_MAX) return false;
                xq += d * qj;
                qj *= F.q;
            }
            // x = x (mod mod), x = xq (mod qk): inverse of mod modulo qk by the
            // extended Euclidean algorithm
            int64_t r0 = (int64_t)F.qk, r1 = (int64_t)(mod % F.qk), s0 = 0, s1 = 1;
            while (r1) {
                int64_t qq = r0 / r1, tmp = r0 - qq * r1;
                r0 = r1; r1 = tmp;
                tmp = s0 - qq * s1; s0 = s1; s1 = tmp;
            }
            uint64_t inv = (uint64_t)((s0 % (int64_t)F.qk + (int64_t)F.qk) % (int64_t)F.qk);
            uint64_t t = (uint64_t)((u128)((xq + F.qk - x % F.qk) % F.qk) * inv % F.qk);
            x += mod * t;
            mod *= F.qk;
        }
        if (powmod(a, x, p) != s) return false;
        *L = x % N;
        return true;
    }
};

bool discrete_log(uint64_t p, uint64_t a, uint64_t s, uint64_t *L)
{
    DlogSolver d(p, a);
    return d.solve(s, L);
}

bool discrete_logs(uint64_t p, uint64_t a, const uint64_t *s, uint64_t count, uint64_t *L)
{
    DlogSolver d(p, a);
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    if (count < 1024) nt = 1;
    std::vector<int> ok(nt, 1);
    auto work = [&](unsigned t) {
        for (uint64_t i = count * t / nt; i < count * (t + 1) / nt; ++i)
            if (!d.solve(s[i], &L[i])) { ok[t] = 0; return; }
    };
    if (nt == 1) work(0);
    else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    for (int v : ok) if (!v) return false;
    return true;
}

// Sliding-window program of exponent e with windows of at most w bits:
// scanning e from its top bit, a zero bit is one more squaring; a one bit
// opens the longest window of <= w bits that ends in a one, and costs that
// many squarings (none for the first window, which initialises x) plus one
// product with the odd power m^v, v the window's value.  Returns the number of
// Montgomery products, table included, or -1 if the program does not fit.
static int build_program(uint64_t e, int w, ExpProg *pg)
{
    memset(pg, 0, sizeof *pg);
    const int L = bitlen(e);
    int i = L - 1, pending = 0, nent = 0, maxidx = 0, products = 0;
    while (i >= 0) {
        if (((e >> i) & 1) == 0) {
            ++pending;
            --i;
            continue;
        }
        int l = i - w + 1 < 0 ? 0 : i - w + 1;
        while (((e >> l) & 1) == 0) ++l;
        const int len = i - l + 1;
        const uint64_t val = (e >> l) & ((1ull << len) - 1);
        const int idx = (int)((val - 1) / 2);
        const int sq = nent == 0 ? 0 : pending + len;
        if (nent >= (int)sizeof pg->ent || sq > 63) return -1;
        pg->ent[nent++] = (uint8_t)(sq | (idx << 6));
        products += sq + (nent > 1 ? 1 : 0);
        if (idx > maxidx) maxidx = idx;
        pending = 0;
        i = l - 1;
    }
    pg->nent = (uint8_t)nent;
    pg->tail = (uint8_t)pending;
    pg->tbl = (uint8_t)(maxidx == 0 ? 1 : maxidx == 1 ? 2 : 4);
    products += pending + (pg->tbl == 1 ? 0 : pg->tbl == 2 ? 2 : 4);
    return products;
}

#ifndef PH_MAX_WINDOW
#define PH_MAX_WINDOW 3
#endif

// The cheapest program over window sizes 1..PH_MAX_WINDOW (at most 3: the
// table holds up to four odd powers).
static ExpProg best_program(uint64_t e)
{
    ExpProg best, cand;
    int best_cost = -1;
    for (int w = 1; w <= PH_MAX_WINDOW && w <= 3; ++w) {
        int c = build_program(e, w, &cand);
        if (c >= 0 && (best_cost < 0 || c < best_cost)) {
            best = cand;
            best_cost = c;
        }
    }
    return best;
}

int program_products(const ExpProg &pg)
{
    int p = (pg.tbl == 1 ? 0 : pg.tbl == 2 ? 2 : 4) + pg.tail + 1;
    for (int k = 1; k < pg.nent; ++k) p += (pg.ent[k] & 63) + 1;
    return p;
}

// Every Montgomery product MP(x, y) = x y R^-1 (R = 2^rbits) multiplies the
// R-powers its operands carry and adds one R^-1.  Started from the plain
// message (power 0), the table holds m2 (power -1), m^3 = MP(m2, m) (-2),
// m^5 = MP(m^3, m2) (-4), m^7 = MP(m^5, m2) (-6); the program leaves
// x = m^e R^alpha, and one more product with K = R^(1-alpha) mod n returns
// m^e.  R has order dividing n-1 mod the prime n, so alpha is tracked mod n-1.
uint64_t mont_exit_constant(uint64_t n, const ExpProg &pg, int rbits)
{
    const uint64_t ord = n - 1;
    auto sub = [&](uint64_t a, uint64_t k) { return (uint64_t)(((u128)a + ord - k % ord) % ord); };
    const uint64_t tpow[4] = {0, sub(0, 2), sub(0, 4), sub(0, 6)};
    uint64_t alpha = tpow[pg.ent[0] >> 6];
    auto square = [&](uint64_t a) { return (uint64_t)(((u128)a * 2 + ord - 1) % ord); };
    for (int k = 1; k < pg.nent; ++k) {
        for (int q = 0; q < (pg.ent[k] & 63); ++q) alpha = square(alpha);
        alpha = sub((uint64_t)(((u128)alpha + tpow[pg.ent[k] >> 6]) % ord), 1);
    }
    for (int q = 0; q < pg.tail; ++q) alpha = square(alpha);
    const uint64_t rmodn = rbits == 32 ? (uint64_t)((1ull << 32) % n)
                                       : (uint64_t)((((u128)1) << 64) % n);
    const uint64_t ex = (uint64_t)(((u128)ord + 1 - alpha) % ord);
    return powmod(rmodn, ex, n);
}

// The 32-bit kernels' program (ExpProg8): for each table size
// T = 1..kProg8MaxTable (odd powers up to 2T - 1; building them costs T products, or 0 for T = 1)
// an exact search over the exponent's bit positions: f[i] is the fewest
// products that leave x = m^(the top i bits of e); the top i bits start x
// when they are an odd value in the table (no product), and otherwise x
// comes from some j < i by i - j squarings and one product with the table
// entry of the low i - j bits of the prefix, which must be odd and in the
// table (a window with its leading zeros).  The low bits only grow as j
// falls, so the search over j stops at the first value above the table.
// e is odd (coprime to the even n - 1), so the last window ends at bit 0.
int program8_products(const ExpProg8 &pg)
{
    int p = (pg.tbl == 1 ? 0 : pg.tbl) + 1;            // table, exit product
    for (int k = 1; k < pg.nent; ++k) p += (pg.ent[k] & 0xFF) + 1;
    return p;
}

ExpProg8 derive_prog8(uint64_t n, uint64_t e)
{
    ExpProg8 best;
    memset(&best, 0, sizeof best);
    const int L = bitlen(e);
    if (L < 1 || L > 32 || !(e & 1)) return best;       // 32-bit exponents only (odd)
    uint64_t pre[33];
    for (int i = 0; i <= L; ++i) pre[i] = i ? e >> (L - i) : 0;
    int best_cost = -1;
    for (int T = 1; T <= kProg8MaxTable; ++T) {
        const uint64_t maxv = 2 * (uint64_t)T - 1;
        int f[33], from[33];
        for (int i = 0; i <= L; ++i) f[i] = -1;
        for (int i = 1; i <= L; ++i) {
            if ((pre[i] & 1) && pre[i] <= maxv) {
                f[i] = 0;
                from[i] = 0;
                continue;
            }
            for (int j = i - 1; j >= 1; --j) {
                const uint64_t v = pre[i] & ((1ull << (i - j)) - 1);
                if (v > maxv) break;
                if (!(v & 1) || f[j] < 0) continue;
                const int c = f[j] + (i - j) + 1;
                if (f[i] < 0 || c < f[i]) {
                    f[i] = c;
                    from[i] = j;
                }
            }
        }
        if (f[L] < 0) continue;
        const int cost = f[L] + (T == 1 ? 0 : T);
        if (best_cost >= 0 && cost >= best_cost) continue;
        // the windows, last to first
        int cuts[33], nc = 0;
        for (int i = L; i > 0; i = from[i]) cuts[nc++] = i;
        if (nc > 32) continue;
        ExpProg8 pg;
        memset(&pg, 0, sizeof pg);
        pg.tbl = (uint8_t)T;
        pg.nent = (uint8_t)nc;
        int prev = 0;
        for (int k = 0; k < nc; ++k) {
            const int i = cuts[nc - 1 - k];
            const uint64_t v = k == 0 ? pre[i] : pre[i] & ((1ull << (i - prev)) - 1);
            pg.ent[k] = (uint16_t)((k == 0 ? 0 : i - prev) | (((v - 1) / 2) << 8));
            prev = i;
        }
        best = pg;
        best_cost = cost;
    }
    // exit constant: table entry k carries R^(-2k) (m^3 = MP(m^2, m), and each
    // next odd power one more product by m^2 = m^2 R^-1); a squaring takes the
    // power a to 2a - 1, a product with entry k to a - 2k - 1
    const uint64_t ord = n - 1;
    auto sub = [&](uint64_t a, uint64_t k) { return (uint64_t)(((u128)a + ord - k % ord) % ord); };
    uint64_t alpha = sub(0, 2 * (uint64_t)(best.ent[0] >> 8));
    for (int k = 1; k < best.nent; ++k) {
        for (int q = 0; q < (best.ent[k] & 0xFF); ++q) alpha = (uint64_t)(((u128)alpha * 2 + ord - 1) % ord);
        alpha = sub(alpha, 2 * (uint64_t)((best.ent[k] >> 8) & 7) + 1);
    }
    const uint64_t rmodn = (uint64_t)((1ull << 32) % n);
    const uint64_t ex = (uint64_t)(((u128)ord + 1 - alpha) % ord);
    best.K = (uint32_t)powmod(rmodn, ex, n);
    best.Kq = best.K * (uint32_t)inv_mod_2_64(n);
    return best;
}

DevInst derive_inst(const phprng_instance &in, int wide, ExpProg *prog)
{
    DevInst d;
    memset(&d, 0, sizeof d);
    d.n = in.n;
    d.e = in.e;
    // e = 2^t + 1: the kernels run the chain of t squarings and one product
    // directly; its program (windows of one bit) has the same exit constant.
    const bool fermat = in.e >= 3 && ((in.e - 1) & (in.e - 2)) == 0;
    d.fermat = fermat ? (uint32_t)(bitlen(in.e - 1) - 1) : 0u;
    d.wide = wide ? 1u : 0u;
    if (fermat)
        build_program(in.e, 1, prog);
    else
        *prog = best_program(in.e);
    if (!wide) {
        const uint32_t ninv32 = (uint32_t)inv_mod_2_64(in.n);
        d.K = mont_exit_constant(in.n, *prog, 32);
        d.ninv = ninv32 | (uint64_t)((uint32_t)d.K * ninv32) << 32;
        uint64_t y = in.n + 1;
        d.ybits = (uint32_t)bitlen(y);
        d.yN = (uint32_t)(y << (32 - d.ybits));
        d.V = (uint64_t)((((u128)1) << 84) / d.yN);
        d.aux = (uint64_t)(((((u128)1) << 95) - 1) / d.yN);
    } else {
        d.ninv = inv_mod_2_64(in.n);
        d.K = mont_exit_constant(in.n, *prog, 64);
        uint64_t r = (uint64_t)((((u128)1) << 64) % in.n);
        d.aux = mulmod(r, r, in.n);
    }
    return d;
}

SkipConst derive_skip(uint64_t p, uint64_t a, int npt)
{
    SkipConst k;
    // The constant skip (a = 1) keeps s_k = s0 for any odd modulus above s0;
    // p = 2 (the unit skip, s0 = 1) is even, and the Montgomery products run
    // modulo 3 instead, with the same values.
    if (a == 1 && p == 2) p = 3;
    uint64_t R = (1ull << 32) % p;
    k.p = (uint32_t)p;
    k.pinv = (uint32_t)inv_mod_2_64(p);
    k.aM = (uint32_t)mulmod(a % p, R, p);
    k.aGM = (uint32_t)mulmod(powmod(a, 32ull * npt, p), R, p);
    k.aMq = k.aM * k.pinv;
    k.aGMq = k.aGM * k.pinv;
    for (int j = 0; j < 32; ++j)
        k.lane[j] = (uint32_t)mulmod(powmod(a, (uint64_t)npt * j, p), R, p);
    return k;
}

SkipConst64 derive_skip64(uint64_t p, uint64_t a, int npt)
{
    SkipConst64 k;
    const uint64_t R = (uint64_t)((((u128)1) << 64) % p);
    k.p = p;
    k.pinv = inv_mod_2_64(p);
    k.aM = mulmod(a % p, R, p);
    k.aGM = mulmod(powmod(a, 32ull * npt, p), R, p);
    k.oneM = R;
    for (int j = 0; j < 32; ++j) k.lane[j] = mulmod(powmod(a, (uint64_t)npt * j, p), R, p);
    return k;
}

SkipTable derive_skip_table(uint64_t p, uint64_t a)
{
    SkipTable t;
    memset(&t, 0, sizeof t);
    if (a == 1) {                                  // constant skip: no cycle, no table
        t.kind = 1;
        t.p = (uint32_t)p;
        return t;
    }
    uint64_t R = (1ull << 32) % p;
    t.p = (uint32_t)p;
    t.pinv = (uint32_t)inv_mod_2_64(p);
    t.aM = (uint32_t)mulmod(a % p, R, p);
    t.oneM = (uint32_t)R;
    t.nT = (p - 1) / kSkipB + 1;
    t.half = (uint64_t)(((u128)p * (p - 1)) / 2);
    for (int l = 0; l < 32; ++l)
        t.laneM[l] = (uint32_t)mulmod(powmod(a, 32ull * l, p), R, p);
    return t;
}

static std::string fmt_inst(const char *what, const phprng_instance &in)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s (n=%llu e=%llu p=%llu a=%llu m0=%llu s0=%llu)", what,
             (unsigned long long)in.n, (unsigned long long)in.e, (unsigned long long)in.p,
             (unsigned long long)in.a, (unsigned long long)in.m0, (unsigned long long)in.s0);
    return buf;
}

int validate_one(int width, const phprng_instance &in, uint32_t flags, std::string *msg)
{
    if (width == 32 && in.n >= (1ull << 32)) {
        *msg = fmt_inst("n does not fit the 32-bit path", in);
        return PHPRNG_EINVAL;
    }
    if (in.n < 5 || !is_prime(in.n)) {
        *msg = fmt_inst("n is not a prime >= 5", in);
        return PHPRNG_ENOTPRIME;
    }
    if ((flags & PHPRNG_REQUIRE_SAFE_PRIME) && !is_prime((in.n - 1) / 2)) {
        *msg = fmt_inst("n is not a safe prime ((n-1)/2 composite)", in);
        return PHPRNG_ENOTPRIME;
    }
    if (in.e < 3 || in.e > in.n - 2 || gcd64(in.e, in.n - 1) != 1) {
        *msg = fmt_inst("e must satisfy 3 <= e <= n-2 and gcd(e, n-1) = 1", in);
        return PHPRNG_EEXPONENT;
    }
    if (in.a == 1) {
        // the constant skip s_k = s0 (Eq. 3 with s_k = b; b = 1, p = 2: the unit skip)
        if (in.p < 2 || in.p >= in.n || in.p >= (1ull << 32) || !is_prime(in.p)) {
            *msg = fmt_inst("constant skip (a = 1): p must be a prime with 2 <= p < n and p < 2^32", in);
            return PHPRNG_ESKIP;
        }
    } else {
        // p < 2^32, or for 64-bit moduli a wide skip prime up to 2^63 (the
        // Implementation section's 63-bit skip generator for 64-bit n)
        const uint64_t pmax = in.n >= (1ull << 32) ? (1ull << 63) : (1ull << 32);
        if (in.p < 3 || in.p >= in.n || in.p >= pmax || !is_prime(in.p)) {
            *msg = fmt_inst("p must be a prime with 3 <= p < n, and p < 2^32 (p < 2^63 when n >= 2^32)", in);
            return PHPRNG_ESKIP;
        }
        if (in.a < 1 || in.a >= in.p || !is_primitive_root(in.a, in.p)) {
            *msg = fmt_inst("a is not a primitive root mod p (a = 1 selects the constant skip)", in);
            return PHPRNG_ESKIP;
        }
    }
    if (in.s0 < 1 || in.s0 >= in.p) {
        *msg = fmt_inst("s0 must lie in [1, p-1]", in);
        return PHPRNG_ESKIP;
    }
    if (in.m0 >= in.n) {
        *msg = fmt_inst("m0 must lie in [0, n)", in);
        return PHPRNG_EINVAL;
    }
    return PHPRNG_OK;
}

int validate_all(int width, const phprng_instance *inst, uint64_t count, uint32_t flags,
                 uint64_t *bad, std::string *msg)
{
    if (width != 0 && width != 32 && width != 64) {
        *msg = "width must be 32, 64 or 0 (mixed)";
        return PHPRNG_EINVAL;
    }
    if (count == 0 || inst == nullptr) {
        *msg = "an instance table with count >= 1 is required";
        return PHPRNG_EINVAL;
    }
    // primality dominates: validate in parallel, report the first failure
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (count < 4096) nt = 1;
    std::vector<int> rc(nt, PHPRNG_OK);
    std::vector<uint64_t> where(nt, UINT64_MAX);
    std::vector<std::string> m(nt);
    auto work = [&](unsigned t) {
        uint64_t lo = count * t / nt, hi = count * (t + 1) / nt;
        for (uint64_t i = lo; i < hi; ++i) {
            int r = validate_one(width, inst[i], flags, &m[t]);
            if (r != PHPRNG_OK) { rc[t] = r; where[t] = i; return; }
        }
    };
    if (nt == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    for (unsigned t = 0; t < nt; ++t) {
        if (rc[t] != PHPRNG_OK) {
            if (bad) *bad = where[t];
            *msg = "instance " + std::to_string(where[t]) + ": " + m[t];
            return rc[t];
        }
    }
    const uint64_t p = inst[0].p, a = inst[0].a;
    for (uint64_t i = 1; i < count; ++i) {
        if (inst[i].p != p || inst[i].a != a) {
            if (bad) *bad = i;
            *msg = "instance " + std::to_string(i) +
                   ": every instance of a context must share one skip generator (p, a)";
            return PHPRNG_ESKIP;
        }
    }
    if (!(flags & PHPRNG_ALLOW_SHARED_N)) {
        std::unordered_set<uint64_t> seen;
        seen.reserve(count * 2);
        for (uint64_t i = 0; i < count; ++i) {
            if (!seen.insert(inst[i].n).second) {
                if (bad) *bad = i;
                *msg = "instance " + std::to_string(i) + ": modulus n=" +
                       std::to_string(inst[i].n) +
                       " repeats an earlier instance (parameter splitting needs distinct n)";
                return PHPRNG_EDUPLICATE;
            }
        }
    }
    return PHPRNG_OK;
}

// ---- seeding -------------------------------------------------------------
namespace {
struct SplitMix64 {
    uint64_t s;
    explicit SplitMix64(uint64_t seed) : s(seed) {}
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    uint64_t below(uint64_t bound) { return (uint64_t)(((u128)next() * bound) >> 64); }
};

bool quick_composite(uint64_t n)
{
    for (uint32_t q : kSmallPrimes)
        if (n % q == 0) return n != q;
    return false;
}

uint64_t next_prime_candidate(SplitMix64 &r, int width, bool safe)
{
    for (;;) {
        uint64_t x = r.next();
        uint64_t n = width == 32 ? ((x >> 33) | (1ull << 31) | 1ull) : (x | (1ull << 63) | 1ull);
        if (quick_composite(n)) continue;
        if (safe && quick_composite((n - 1) / 2)) continue;
        if (!is_prime(n)) continue;
        if (safe && !is_prime((n - 1) / 2)) continue;
        return n;
    }
}
}  // namespace

int draw_instances(int width, uint64_t count, uint64_t seed, uint32_t flags,
                   phprng_instance *out, std::string *msg)
{
    if (width != 32 && width != 64) {
        *msg = "phprng_draw_instances: width must be 32 or 64";
        return PHPRNG_EINVAL;
    }
    if (count == 0 || out == nullptr) {
        *msg = "phprng_draw_instances: count >= 1 and an output table are required";
        return PHPRNG_EINVAL;
    }
    const bool safe = (flags & PHPRNG_REQUIRE_SAFE_PRIME) != 0;
    const uint64_t p = 2147483647ull, a = 784588716ull;
    // Instance i draws from its own SplitMix64 stream, seeded by output i of
    // the master stream, so the table does not depend on the thread count.
    std::vector<uint64_t> iseed(count);
    {
        SplitMix64 master(seed);
        for (uint64_t i = 0; i < count; ++i) iseed[i] = master.next();
    }
    std::vector<SplitMix64> rng;
    rng.reserve(count);
    for (uint64_t i = 0; i < count; ++i) rng.emplace_back(iseed[i]);
    std::vector<uint64_t> ns(count);
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    if (count < 256) nt = 1;
    auto work = [&](unsigned t) {
        for (uint64_t i = count * t / nt; i < count * (t + 1) / nt; ++i)
            ns[i] = next_prime_candidate(rng[i], width, safe);
    };
    if (nt == 1) work(0);
    else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    // distinct moduli: a later instance that repeats an earlier modulus keeps
    // drawing from its own stream (sequential, hence deterministic)
    std::unordered_set<uint64_t> seen;
    seen.reserve(count * 2);
    for (uint64_t i = 0; i < count; ++i) {
        while (!seen.insert(ns[i]).second) ns[i] = next_prime_candidate(rng[i], width, safe);
    }
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t n = ns[i];
        SplitMix64 &r = rng[i];
        uint64_t e;
        do { e = 3 + r.below(n - 4); } while (gcd64(e, n - 1) != 1);   // e in [3, n-2]
        uint64_t m0 = r.below(n);
        uint64_t L = r.below(p - 1);
        out[i].n = n; out[i].e = e; out[i].p = p; out[i].a = a;
        out[i].m0 = m0;
        out[i].s0 = powmod(a, L, p);
    }
    return PHPRNG_OK;
}

}  // namespace phprng
