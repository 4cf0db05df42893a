"""CPU checks of the library's own arithmetic, compiled for the host from the
same source the kernels use (arith.cuh, hostnt.cpp): Montgomery
exponentiation with the exit constant K, the integer-built R, the skip
constants and the discrete log, against Python's pow and IEEE division."""
import ctypes
import os
import random
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from conftest import ROOT

P31, A31 = 2147483647, 784588716


@pytest.fixture(scope="module")
def h(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("harness") / "host_arith.so")
    subprocess.check_call([
        "g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
        os.path.join(ROOT, "tests", "harness", "host_arith.cpp"),
        os.path.join(ROOT, "paper_1411_2484_gb300", "csrc", "hostnt.cpp"),
        "-o", out, "-lpthread"])
    lib = ctypes.CDLL(out)
    P64 = ctypes.POINTER(ctypes.c_uint64)
    u64 = ctypes.c_uint64
    lib.h_real32_many.argtypes = [P64, P64, ctypes.POINTER(ctypes.c_double), u64]
    lib.h_modexp_many.argtypes = [P64, P64, P64, P64, u64, ctypes.c_int]
    lib.h_skip_step.restype = u64
    lib.h_skip_step.argtypes = [u64, u64, u64]
    lib.h_skip_lane.restype = u64
    lib.h_skip_lane.argtypes = [u64, u64, u64, ctypes.c_int, ctypes.c_int]
    lib.h_discrete_log.argtypes = [u64, u64, u64, P64]
    lib.h_addmod.restype = u64
    lib.h_addmod.argtypes = [u64, u64, u64, ctypes.c_int]
    lib.h_real32_fast_many.argtypes = [P64, P64, ctypes.POINTER(ctypes.c_double), u64]
    lib.h_real32_split_many.argtypes = [P64, P64, ctypes.POINTER(ctypes.c_double), u64]
    lib.h_modexp8_many.argtypes = [P64, P64, P64, P64, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64), u64]
    lib.h_real32_fast_frac.restype = ctypes.c_uint32
    lib.h_prog8_words.argtypes = [u64, u64, ctypes.POINTER(ctypes.c_uint32)]
    lib.h_real32_fast_frac.argtypes = [u64, u64]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def modexp(h, m, e, n, wide):
    m, e, n = (np.ascontiguousarray(x, dtype=np.uint64) for x in (m, e, n))
    out = np.empty_like(m)
    h.h_modexp_many(_p(m), _p(e), _p(n), _p(out), m.size, wide)
    return out


def test_real32_equals_ieee_division(h):
    rng = np.random.default_rng(1)
    k = 400000
    n = np.concatenate([rng.integers(3, 1 << 32, k // 2, dtype=np.uint64) | np.uint64(1),
                        rng.integers(3, 5000, k // 2, dtype=np.uint64) | np.uint64(1)])
    n = np.minimum(n, np.uint64((1 << 32) - 5))
    c = (rng.integers(0, 1 << 62, k, dtype=np.uint64) % n).astype(np.uint64)
    c[::7] = n[::7] - np.uint64(1)
    c[::11] = 0
    out = np.empty(k, dtype=np.float64)
    h.h_real32_many(_p(n), _p(c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), k)
    ref = (c + np.uint64(1)).astype(np.float64) / (n + np.uint64(1)).astype(np.float64)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
    for i in range(0, k, 997):            # and against exact rationals
        assert out[i] == float(Fraction(int(c[i]) + 1, int(n[i]) + 1))


def test_real32_every_c_for_small_moduli(h):
    for nn in (3, 5, 7, 23, 31, 127, 255, 257, 1023, 4093, 8191):
        c = np.arange(nn, dtype=np.uint64)
        n = np.full(nn, nn, dtype=np.uint64)
        out = np.empty(nn, dtype=np.float64)
        h.h_real32_many(_p(n), _p(c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nn)
        for ci in range(nn):
            assert out[ci] == float(Fraction(ci + 1, nn + 1))


@pytest.mark.parametrize("wide", [0, 1])
def test_montgomery_exponentiation_matches_pow(h, wide):
    from paper_1411_2484_gb300 import workloads
    rng = random.Random(2 + wide)
    ns = [4294967291, 4294967087, 2147483659, 23, 101, 65537] if not wide else \
        [18446744073709551557, 9223372036854775837, 4294967291, 23]
    ns += [int(x) for x in workloads.draw_instances(20, width=64 if wide else 32, seed=3)["n"]]
    ms, es, nn, ref = [], [], [], []
    for n in ns:
        for _ in range(300):
            e = rng.randrange(3, n - 1) if n > 5 else 3
            m = rng.choice([0, 1, n - 1, rng.randrange(n)])
            ms.append(m); es.append(e); nn.append(n); ref.append(pow(m, e, n))
        for e in (3, 5, 9, 17, n - 2):
            m = rng.randrange(n)
            ms.append(m); es.append(e); nn.append(n); ref.append(pow(m, e, n))
    out = modexp(h, ms, es, nn, wide)
    assert [int(x) for x in out] == ref


def test_heavy_programs_match_pow_and_save_products(h):
    """The 32-bit kernels' programs (exact search over table sizes 1..6)
    give m^e mod n for random 32-bit primes and exponents, the paper's small
    exponents and extreme ones, and never need more products than the
    standard sliding-window program (about 0.6 fewer on average)."""
    rng = random.Random(31)
    primes = []
    while len(primes) < 40:
        q = rng.randrange((1 << 31) + 1, 1 << 32) | 1
        if pow(2, q - 1, q) == 1 and pow(3, q - 1, q) == 1 and pow(5, q - 1, q) == 1:
            primes.append(q)
    import math
    ms, es, ns = [], [], []
    for q in primes:
        for _ in range(40):
            e = rng.randrange(3, q - 1)
            while math.gcd(e, q - 1) != 1:
                e = rng.randrange(3, q - 1)
            ms.append(rng.randrange(0, q)); es.append(e); ns.append(q)
        for e in (3, 5, 7, 9, 17, 65537, 0xFFFFFFFF & (q - 2)):
            if math.gcd(e, q - 1) == 1 and e < q - 1:
                for mm in (0, 1, 2, q - 1):
                    ms.append(mm); es.append(e); ns.append(q)
    m = np.array(ms, dtype=np.uint64); e = np.array(es, dtype=np.uint64); n = np.array(ns, dtype=np.uint64)
    out = np.empty_like(m)
    p8 = np.empty(m.size, dtype=np.int64)
    p4 = np.empty(m.size, dtype=np.int64)
    h.h_modexp8_many(_p(m), _p(e), _p(n), _p(out), p8.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     p4.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), m.size)
    want = np.array([pow(int(a), int(b), int(c)) for a, b, c in zip(m, e, n)], dtype=np.uint64)
    assert np.array_equal(out, want)
    assert np.all(p8 <= p4)
    assert 0.3 < float((p4 - p8).mean()) < 1.2


def test_exact_search_is_minimal_over_all_window_cuts(h):
    """For every odd exponent below 2^10, and for 15- and 16-bit exponents
    whose best table has 6 entries, the program's product count equals the
    minimum over all ways of cutting the exponent's bits into windows (brute
    force over every subset of cut positions), each window an odd value of at
    most 2T - 1 after its leading zeros, for table sizes T = 1..6: the first
    window loads a table entry, each later one costs its length in squarings
    plus one product; the table costs T products for T >= 2 (m^2 and T - 1
    steps), and the exit product one more."""
    def brute(e):
        # least cost of the windows for each table size T = 1..6
        bits = bin(e)[2:]
        L, best = len(bits), [None] * 7
        for mask in range(1 << (L - 1)):
            cuts = [0] + [k + 1 for k in range(L - 1) if mask >> k & 1] + [L]
            segs = [bits[a:b] for a, b in zip(cuts, cuts[1:])]
            vals = [int(sg, 2) for sg in segs]
            if any(v % 2 == 0 for v in vals) or max(vals) > 11:
                continue
            cost = sum(len(sg) + 1 for sg in segs[1:])
            for T in range((max(vals) + 1) // 2, 7):      # every table that holds the windows
                if best[T] is None or cost < best[T]:
                    best[T] = cost
        return 1 + min(best[T] + (T if T >= 2 else 0) for T in range(1, 7) if best[T] is not None)
    # a 6-entry table is strictly best for these (one product fewer than 5)
    wide = [22987, 19851, 45639]
    es = np.array(list(range(3, 1024, 2)) + wide, dtype=np.uint64)
    n = np.full(es.size, 4294967291, dtype=np.uint64)
    m = np.full(es.size, 12345, dtype=np.uint64)
    out = np.empty_like(m)
    p8 = np.empty(es.size, dtype=np.int64)
    p4 = np.empty(es.size, dtype=np.int64)
    h.h_modexp8_many(_p(m), _p(es), _p(n), _p(out), p8.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     p4.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), es.size)
    for e, got, x in zip(es, p8, out):
        assert int(got) == brute(int(e)), (int(e), int(got))
        assert int(x) == pow(12345, int(e), 4294967291)


def test_exact_search_programs_index_inside_their_table(h):
    """Every window of a program reads a table entry the program builds (index
    below its table size, at most 6 entries: the 6 KiB per warp the kernels
    reserve), there are 1 to 32 windows, every window after the first has at
    least one squaring, and the windows' bits add up to the exponent's length:
    random 32-bit exponents and the extreme ones."""
    rng = random.Random(77)
    n = 4294967291
    es = [3, 5, 9, 17, 65537, 0x55555555, 0xAAAAAAAB, 0xFFFFFFFD, (1 << 31) + 1, n - 2]
    es += [rng.randrange(3, 1 << 32) | 1 for _ in range(3000)]
    w = (ctypes.c_uint32 * 66)()
    for e in es:
        h.h_prog8_words(n, e, w)
        tbl, nent = w[0], w[1]
        assert 1 <= tbl <= 6 and 1 <= nent <= 32, (e, tbl, nent)
        sq = [w[2 + k] for k in range(nent)]
        idx = [w[34 + k] for k in range(nent)]
        assert all(i < tbl for i in idx), (e, tbl, idx)
        assert all(q >= 1 for q in sq[1:]), (e, sq)
        first_bits = (2 * idx[0] + 1).bit_length()
        assert first_bits + sum(sq[1:]) == e.bit_length(), (e, sq, idx)


def test_skip_constants(h):
    rng = random.Random(4)
    for p, a in ((P31, A31), (11, 2), (4294967291, 2), (101, 2)):
        for _ in range(200):
            s = rng.randrange(1, p)
            assert h.h_skip_step(s, p, a) == a * s % p
            npt, lane = rng.choice([1, 2, 4, 8]), rng.randrange(33)
            expo = npt * lane if lane < 32 else 32 * npt
            assert h.h_skip_lane(s, p, a, npt, lane) == s * pow(a, expo, p) % p


def test_addmod(h):
    rng = random.Random(5)
    for wide, bits in ((0, 32), (1, 64)):
        for _ in range(2000):
            n = rng.randrange(3, 1 << bits)
            a, b = rng.randrange(n), rng.randrange(n)
            assert h.h_addmod(a, b, n, wide) == (a + b) % n


def test_discrete_log(h):
    rng = random.Random(6)
    L = ctypes.c_uint64()
    for p, a in ((P31, A31), (11, 2), (1000003, 2), (4294967291, 2)):
        for _ in range(50):
            s = rng.randrange(1, p)
            assert h.h_discrete_log(p, a, s, ctypes.byref(L)) == 1
            assert pow(a, L.value, p) == s and L.value < p - 1


def test_u128_to_double_is_correctly_rounded(h):
    h.h_u128_to_double_many.argtypes = [ctypes.POINTER(ctypes.c_uint64)] * 2 + [
        ctypes.POINTER(ctypes.c_double), ctypes.c_uint64]
    rng = random.Random(7)
    vals = [0, 1, (1 << 64) - 1, 1 << 64, (1 << 128) - 1, (1 << 53) + 1, (1 << 117) + (1 << 64)]
    for _ in range(20000):
        bits = rng.randrange(1, 129)
        v = rng.getrandbits(bits)
        vals.append(v)
        # halfway cases and their neighbours
        if bits > 60:
            k = bits - 54
            base = (v >> k) << k
            vals += [base + (1 << (k - 1)), base + (1 << (k - 1)) - 1, base + (1 << (k - 1)) + 1]
    vals = [v for v in vals if v < (1 << 128)]
    hi = np.array([v >> 64 for v in vals], dtype=np.uint64)
    lo = np.array([v & ((1 << 64) - 1) for v in vals], dtype=np.uint64)
    out = np.empty(len(vals), dtype=np.float64)
    h.h_u128_to_double_many(_p(hi), _p(lo), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            len(vals))
    for v, o in zip(vals, out):
        assert o == float(v), v          # Python int -> float rounds to nearest even


def test_hist_bin_matches_floor(h):
    h.h_hist_bin_many.argtypes = [ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint64]
    rng = np.random.default_rng(8)
    r = np.concatenate([rng.random(100000), [0.0, 1.0, 0.5, 255 / 256, np.nextafter(1.0, 0.0),
                                               1 / 256, np.nextafter(1 / 256, 0.0), 2.0 ** -60]])
    out = np.empty(r.size, dtype=np.uint32)
    h.h_hist_bin_many(r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), r.size)
    ref = np.minimum(np.floor(r * 256.0), 255).astype(np.uint32)
    assert np.array_equal(out, ref)


def test_hist_bin_integer_equals_floor(h):
    """The fused mode's integer bin equals floor(256 (c+1)/(n+1)), exact
    multiples of 1/256 and tiny moduli included."""
    h.h_hist_bin_int_many.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint64]
    rng = np.random.default_rng(21)
    k = 200000
    n = np.concatenate([rng.integers(3, 1 << 32, k // 2, dtype=np.uint64) | np.uint64(1),
                        rng.integers(3, 3000, k // 2, dtype=np.uint64) | np.uint64(1)])
    n = np.minimum(n, np.uint64((1 << 32) - 5))
    c = (rng.integers(0, 1 << 62, k, dtype=np.uint64) % n).astype(np.uint64)
    c[::5] = n[::5] - np.uint64(1)
    c[::9] = 0
    # (c+1)/(n+1) exactly k'/256: n+1 = 256 t, c+1 = k' t
    ex_n, ex_c = [], []
    rr = random.Random(22)
    while len(ex_n) < 4000:
        t = rr.randrange(1, 1 << 24)
        nn = 256 * t - 1
        kk = rr.randrange(1, 256)
        ex_n.append(nn)
        ex_c.append(kk * t - 1)
        ex_n.append(nn)
        ex_c.append(kk * t - 2 if kk * t >= 2 else 0)
    for nn in (3, 7, 31, 127, 8191, 131071, 524287):      # n + 1 a power of two
        for cc in range(0, nn, max(1, nn // 300)):
            ex_n.append(nn)
            ex_c.append(cc)
    n = np.concatenate([n, np.array(ex_n, dtype=np.uint64)])
    c = np.concatenate([c, np.array(ex_c, dtype=np.uint64)])
    out = np.empty(n.size, dtype=np.uint32)
    P64 = ctypes.POINTER(ctypes.c_uint64)
    h.h_hist_bin_int_many(n.ctypes.data_as(P64), c.ctypes.data_as(P64),
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n.size)
    ref = np.array([(256 * (int(ci) + 1)) // (int(ni) + 1) for ni, ci in zip(n, c)], dtype=np.uint32)
    bad = np.flatnonzero(out != ref)
    assert bad.size == 0, (n[bad[0]], c[bad[0]], out[bad[0]], ref[bad[0]])


@pytest.mark.parametrize("form", ["h_real32_fast_many", "h_real32_split_many"])
def test_real32_fast_equals_ieee_division(h, form):
    """The fast rounding decision, and its exact fallback band (forced); in
    one function, and as the branch-free estimate plus the exact decision for
    the inputs it flags."""
    rng = np.random.default_rng(11)
    k = 600000
    n = np.concatenate([rng.integers(3, 1 << 32, k // 2, dtype=np.uint64) | np.uint64(1),
                        rng.integers(3, 5000, k // 2, dtype=np.uint64) | np.uint64(1)])
    n = np.minimum(n, np.uint64((1 << 32) - 5))
    c = (rng.integers(0, 1 << 62, k, dtype=np.uint64) % n).astype(np.uint64)
    c[::7] = n[::7] - np.uint64(1)
    c[::11] = 0
    # add inputs whose estimate lands in the fallback band 1021 <= f < 1024
    band_n, band_c = [], []
    rr = random.Random(12)
    while len(band_n) < 3000:
        nn = rr.randrange(3, (1 << 32) - 5) | 1
        cc = rr.randrange(nn)
        if 1018 <= h.h_real32_fast_frac(nn, cc) < 1028:
            band_n.append(nn)
            band_c.append(cc)
    n = np.concatenate([n, np.array(band_n, dtype=np.uint64)])
    c = np.concatenate([c, np.array(band_c, dtype=np.uint64)])
    out = np.empty(n.size, dtype=np.float64)
    getattr(h, form)(_p(n), _p(c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.size)
    ref = (c + np.uint64(1)).astype(np.float64) / (n + np.uint64(1)).astype(np.float64)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
    for nn in (3, 5, 7, 23, 31, 127, 255, 257, 4093, 8191, 2147483647):   # every c, small n
        if nn > 10000:
            cs = np.array([0, 1, nn - 2, nn - 1] + [rr.randrange(nn) for _ in range(5000)],
                          dtype=np.uint64)
        else:
            cs = np.arange(nn, dtype=np.uint64)
        ns = np.full(cs.size, nn, dtype=np.uint64)
        o = np.empty(cs.size, dtype=np.float64)
        getattr(h, form)(_p(ns), _p(cs), o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             cs.size)
        assert all(o[i] == float(Fraction(int(cs[i]) + 1, nn + 1)) for i in range(cs.size))
