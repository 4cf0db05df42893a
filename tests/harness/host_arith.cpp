// Host build of the library's hot-path arithmetic (arith.cuh) and instance
// layer (hostnt.cpp) for CPU tests: the same source the kernels compile,
// instantiated with one number per lane.
#include <cstdint>
#include "../../paper_1411_2484_gb300/csrc/internal.h"

using namespace phprng;

extern "C" {

void h_real32_many(const uint64_t *n, const uint64_t *c, double *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) {
        phprng_instance in{n[i], 3, 3, 2, 0, 1};
        ExpProg pg;
        DevInst d = derive_inst(in, 0, &pg);
        out[i] = real32((uint32_t)c[i], d.yN, d.ybits, d.V);
    }
}

void h_real32_fast_many(const uint64_t *n, const uint64_t *c, double *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) {
        phprng_instance in{n[i], 3, 3, 2, 0, 1};
        ExpProg pg;
        DevInst d = derive_inst(in, 0, &pg);
        out[i] = real32_fast((uint32_t)c[i], d.yN, d.ybits, d.aux);
    }
}

// R by the branch-free estimate and, for inputs it flags, the exact decision
// (the form the generator uses for two numbers at a time)
void h_real32_split_many(const uint64_t *n, const uint64_t *c, double *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) {
        phprng_instance in{n[i], 3, 3, 2, 0, 1};
        ExpProg pg;
        DevInst d = derive_inst(in, 0, &pg);
        uint32_t amb;
        out[i] = real32_est((uint32_t)c[i], d.yN, d.ybits, d.aux, &amb);
        if (amb) out[i] = real32_exact((uint32_t)c[i], d.yN, d.ybits, d.aux);
    }
}

// m^e mod n by the exact-search program (tables of up to kProg8MaxTable odd powers);
// *products_out[i] gets its Montgomery products and std_out[i] those of the
// standard program, for the comparison
void h_modexp8_many(const uint64_t *m, const uint64_t *e, const uint64_t *n, uint64_t *out,
                    int64_t *products8, int64_t *products, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) {
        phprng_instance in{n[i], e[i], 3, 2, 0, 1};
        ExpProg pg;
        derive_inst(in, 0, &pg);
        const ExpProg8 p8 = derive_prog8(n[i], e[i]);
        uint32_t msg[1] = {(uint32_t)m[i]}, x[1];
        modexp_prog8<1>(x, msg, p8, (uint32_t)n[i], (uint32_t)inv_mod_2_64(n[i]));
        out[i] = x[0];
        products8[i] = program8_products(p8);
        products[i] = program_products(pg);
    }
}

// fraction bits f of the fast quotient estimate, to find inputs in the band
// where real32_fast falls back to the exact remainder
// The exact-search program of (n, e) as plain words: out[0] table size,
// out[1] windows, out[2 + k] window k's squarings and out[34 + k] its table
// index (k < 32), for checks of the layout the kernels index by.
void h_prog8_words(uint64_t n, uint64_t e, uint32_t *out)
{
    const ExpProg8 p8 = derive_prog8(n, e);
    out[0] = p8.tbl;
    out[1] = p8.nent;
    for (int k = 0; k < 32; ++k) {
        out[2 + k] = p8.ent[k] & 0xFF;
        out[34 + k] = (p8.ent[k] >> 8) & 0xFF;
    }
}

uint32_t h_real32_fast_frac(uint64_t n, uint64_t c)
{
    phprng_instance in{n, 3, 3, 2, 0, 1};
    ExpProg pg;
    DevInst d = derive_inst(in, 0, &pg);
    uint32_t x = (uint32_t)c + 1;
    int xb = 32 - clz32(x);
    uint32_t A = x << (32 - xb);
    uint32_t extra = A < d.yN ? 1u : 0u;
    const uint64_t P = (uint64_t)A * (uint32_t)d.aux;
    const uint64_t H = (uint64_t)A * (uint32_t)(d.aux >> 32);
    const uint64_t Xf = (H << extra) + (P >> (32 - extra));
    return (uint32_t)Xf & 0x7FFu;
}

void h_modexp_many(const uint64_t *m, const uint64_t *e, const uint64_t *n, uint64_t *out,
                   uint64_t count, int wide)
{
    for (uint64_t i = 0; i < count; ++i) {
        phprng_instance in{n[i], e[i], 3, 2, 0, 1};
        ExpProg pg;
        DevInst d = derive_inst(in, wide, &pg);
        if (!wide) {
            uint32_t msg[1] = {(uint32_t)m[i]}, x[1];
            modexp_prog<1, uint32_t>(x, msg, pg, (uint32_t)d.n, (uint32_t)d.ninv, (uint32_t)d.K,
                                     (uint32_t)(d.ninv >> 32));
            out[i] = x[0];
        } else {
            uint64_t msg[1] = {m[i]}, x[1];
            modexp_prog<1, uint64_t>(x, msg, pg, d.n, d.ninv, d.K, 0);
            out[i] = x[0];
        }
    }
}

// One skip step s -> a s mod p through the Montgomery constants the kernels use.
uint64_t h_skip_step(uint64_t s, uint64_t p, uint64_t a)
{
    SkipConst k = derive_skip(p, a, 4);
    const uint32_t r = mont32c((uint32_t)s, k.aM, k.aMq, k.p);
    return r == mont32((uint32_t)s, k.aM, k.p, k.pinv) ? r : ~0ull;
}

// s a^(npt*lane) mod p and s a^(32*npt) mod p from the lane constants.
uint64_t h_skip_lane(uint64_t s, uint64_t p, uint64_t a, int npt, int lane)
{
    SkipConst k = derive_skip(p, a, npt);
    if (lane == 32) return mont32c((uint32_t)s, k.aGM, k.aGMq, k.p);
    return mont32((uint32_t)s, k.lane[lane], k.p, k.pinv);
}

int h_discrete_log(uint64_t p, uint64_t a, uint64_t s, uint64_t *L)
{
    return discrete_log(p, a, s, L) ? 1 : 0;
}

uint64_t h_addmod(uint64_t a, uint64_t b, uint64_t n, int wide)
{
    return wide ? addmod64(a, b, n) : addmod32((uint32_t)a, (uint32_t)b, (uint32_t)n);
}
}

extern "C" {
void h_u128_to_double_many(const uint64_t *hi, const uint64_t *lo, double *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) out[i] = u128_to_double(hi[i], lo[i]);
}

void h_hist_bin_many(const double *r, uint32_t *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) out[i] = hist_bin256(r[i]);
}

// floor(256 (c+1)/(n+1)) the integer way, with the per-instance constants
// derived as the library derives them.
void h_hist_bin_int_many(const uint64_t *n, const uint64_t *c, uint32_t *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i) {
        phprng_instance in{n[i], 3, 2, 1, 0, 1};
        ExpProg pg;
        const DevInst d = derive_inst(in, 0, &pg);
        out[i] = hist_bin256_int((uint32_t)c[i], d.yN, d.ybits, (uint32_t)(d.V >> 44));
    }
}
}
