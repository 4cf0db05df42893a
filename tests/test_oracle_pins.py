"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: Python's
own big-integer pow and exact rational division, brute force on tiny
moduli, closed forms, theorems the paper states (Fermat, Eq. 2 decryption,
the period n(p-1) and the (p-1)-fold multiplicity of every ciphertext), and
printed values (Fig. 2, Fig. 3, a hand-worked Eq. 9 table).
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden

P31, A31 = 2147483647, 784588716


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def primitive_root(p):
    phi = p - 1
    fac, x, d = set(), phi, 2
    while d * d <= x:
        while x % d == 0:
            fac.add(d)
            x //= d
        d += 1
    if x > 1:
        fac.add(x)
    for g in range(2, p):
        if all(pow(g, phi // q, p) != 1 for q in fac):
            return g
    return 1  # p = 2


def small_primes(lo, hi):
    return [q for q in range(max(lo, 2), hi) if all(q % d for d in range(2, int(q ** 0.5) + 1))]


# ------------------------------------------------------------ modular arithmetic
def test_mulmod_powmod_match_python_pow(oracle_mod):
    rng = random.Random(1)
    for bits_n in (5, 16, 31, 32, 33, 48, 63, 64):
        for _ in range(300):
            n = rng.randrange(2, 1 << bits_n) | 1
            x, y = rng.randrange(n), rng.randrange(n)
            e = rng.randrange(1 << rng.randrange(1, 65))
            assert oracle_mod.mulmod(x, y, n) == x * y % n
            assert oracle_mod.powmod(x, e, n) == pow(x, e, n)
    assert oracle_mod.powmod(5, 0, 7) == 1


def test_fermat_little_theorem(oracle_mod):
    """For prime n and m in (Z/nZ)*: m^(n-1) mod n = 1 (Introduction, Eq. 2)."""
    rng = random.Random(2)
    for n in (23, 4294967087, 4294967291, 18446744073709551557):
        for _ in range(200):
            m = rng.randrange(1, n)
            assert oracle_mod.powmod(m, n - 1, n) == 1


def test_fig3_key_decrypts(oracle_mod):
    """Eq. 2 with the Fig. 3 key: c^d mod n recovers every message."""
    h, _ = read_golden("fig3_key.txt")
    n, e, d = int(h["n"]), int(h["e"]), int(h["d"])
    assert (d * e) % (n - 1) == 1
    rng = random.Random(3)
    for m in [0, 1, 2, n - 2, n - 1] + [rng.randrange(n) for _ in range(2000)]:
        c = oracle_mod.powmod(m, e, n)
        assert oracle_mod.powmod(c, d, n) == m


def test_decryption_random_64bit_keys(oracle_mod):
    rng = random.Random(4)
    for n in (18446744073709551557, 9223372036854775837):
        for _ in range(50):
            e = rng.randrange(3, n - 1)
            if math.gcd(e, n - 1) != 1:
                continue
            d = pow(e, -1, n - 1)
            m = rng.randrange(n)
            assert oracle_mod.powmod(oracle_mod.powmod(m, e, n), d, n) == m


def test_encryption_is_a_bijection_on_tiny_primes(oracle_mod):
    """x -> x^e mod n permutes Z/nZ for every allowed e (Introduction)."""
    for n in small_primes(5, 90):
        for e in range(3, n - 1):
            images = {oracle_mod.powmod(x, e, n) for x in range(n)}
            if math.gcd(e, n - 1) == 1:
                assert images == set(range(n)), (n, e)
            else:
                assert len(images) < n, (n, e)


def test_reflection_symmetry(oracle_mod):
    """(n-m)^e mod n = n - (m^e mod n) for odd e (Message skipping algorithms)."""
    rng = random.Random(5)
    for n in (4294967087, 2147483659, 18446744073709551557):
        for _ in range(300):
            e = rng.randrange(3, n - 1) | 1
            m = rng.randrange(1, n)
            assert oracle_mod.powmod(n - m, e, n) == n - oracle_mod.powmod(m, e, n)


def test_constant_skip_identity(oracle_mod):
    """Eq. 4: (k b)^e mod n = ((b^e mod n)(k^e mod n)) mod n."""
    rng = random.Random(6)
    n = 4294967087
    for _ in range(300):
        b, k, e = rng.randrange(2, n - 1), rng.randrange(n), rng.randrange(3, n - 1)
        lhs = oracle_mod.powmod(oracle_mod.mulmod(k, b, n), e, n)
        rhs = oracle_mod.mulmod(oracle_mod.powmod(b, e, n), oracle_mod.powmod(k, e, n), n)
        assert lhs == rhs


# ------------------------------------------------------------ Eq. 9 generator
def test_hand_worked_eq9_table(oracle_mod):
    h, rows = read_golden("tiny_n23_eq9.txt")
    n, e, p, a = (int(h[k]) for k in ("n", "e", "p", "a"))
    m, s = int(h["m0"]), int(h["s0"])
    for k, sk, mk, ck, num, den in rows:
        c, r, (m, s) = oracle_mod.generate(n, e, p, a, m, s, 1)
        assert (s, m, int(c[0])) == (sk, mk, ck), k
        assert r[0] == num / den
        assert bits(r[0]) == bits(float(Fraction(num, den)))


def test_fig2_unit_skip_cribs(oracle_mod):
    """Unit skip s_k = 1 is the skip generator with p = 2, a = 1 (s = 1*1 mod 2)."""
    h, rows = read_golden("fig2_unit_skip.txt")
    n, e = int(h["n"]), int(h["e"])
    c, _, _ = oracle_mod.generate(n, e, 2, 1, n - 1, 1, len(rows))   # m_1 = 0
    assert [int(x) for x in c] == [row[1] for row in rows]


TINY = [  # (n, p, e): p < n, both prime
    (23, 11, 3), (47, 23, 5), (59, 29, 3), (83, 41, 13), (107, 53, 5), (29, 13, 3),
    (37, 31, 5), (101, 97, 3), (13, 11, 5), (11, 7, 3),
]


@pytest.mark.parametrize("n,p,e", TINY)
def test_period_and_uniform_full_period(oracle_mod, n, p, e):
    """Period P = n(p-1); over it every ciphertext appears exactly p-1 times
    (Message skipping algorithms, proof after Eq. 6)."""
    assert math.gcd(e, n - 1) == 1
    a = primitive_root(p)
    rng = random.Random(n * 1000 + p)
    m0, s0 = rng.randrange(n), rng.randrange(1, p)
    P = n * (p - 1)
    # walk the state and find the first return
    m, s = m0, s0
    first_return = None
    c_all = []
    for k in range(1, P + 1):
        c, _, (m, s) = oracle_mod.generate(n, e, p, a, m, s, 1)
        c_all.append(int(c[0]))
        if (m, s) == (m0, s0) and first_return is None:
            first_return = k
    assert first_return == P
    counts = np.bincount(np.array(c_all), minlength=n)
    assert np.all(counts == p - 1)
    # bulk call gives the same stream
    c_bulk, _, st = oracle_mod.generate(n, e, p, a, m0, s0, P)
    assert [int(x) for x in c_bulk] == c_all and st == (m0, s0)


def test_real_32bit_is_correctly_rounded(oracle_mod):
    rng = random.Random(7)
    ns = [4294967291, 4294967087, 2147483659, 23, 3, 5, 8191]
    for n in ns:
        cs = [0, 1, n - 1, n - 2, (n - 1) // 2] + [rng.randrange(n) for _ in range(2000)]
        cs += [(1 << j) - 1 for j in range(1, 32) if (1 << j) - 1 < n]
        for c in cs:
            r = oracle_mod.real(c, n)
            assert bits(r) == bits(float(Fraction(c + 1, n + 1)))
            assert 0.0 < r < 1.0


def test_real_64bit_reading(oracle_mod):
    """64-bit n: RN(RN(c+1) / RN(n+1)) -- each operand rounded to double first."""
    rng = random.Random(8)
    n = 18446744073709551557
    differs = 0
    for _ in range(5000):
        c = rng.randrange(n)
        r = oracle_mod.real(c, n)
        assert bits(r) == bits(float(c + 1) / float(n + 1))
        differs += bits(r) != bits(float(Fraction(c + 1, n + 1)))
    assert differs > 0            # the reading is not the exact-rational rounding
    assert oracle_mod.real(n - 1, n) == 1.0   # R can reach 1.0 for 64-bit n


# ------------------------------------------------------------ Eq. 7 skip-ahead
@pytest.mark.parametrize("n,p,e", TINY[:5])
def test_skip_stepping_matches_generation_tiny(oracle_mod, n, p, e):
    a = primitive_root(p)
    rng = random.Random(p)
    for _ in range(40):
        m, s = rng.randrange(n), rng.randrange(1, p)
        k = rng.randrange(0, 5 * n * (p - 1))
        _, _, st = oracle_mod.generate(n, e, p, a, m, s, k)
        assert oracle_mod.skip_stepping(n, p, a, m, s, k) == st


def test_skip_stepping_matches_generation_32bit(oracle_mod):
    rng = random.Random(9)
    n, e = 4294967087, 9
    for _ in range(20):
        m, s = rng.randrange(n), rng.randrange(1, P31)
        k = rng.randrange(0, 200000)
        _, _, st = oracle_mod.generate(n, e, P31, A31, m, s, k)
        assert oracle_mod.skip_stepping(n, P31, A31, m, s, k) == st


@pytest.mark.parametrize("p", [11, 13, 23, 29, 101, 257])
def test_prefix_table_tiny(oracle_mod, p):
    a = primitive_root(p)
    for stride in (1, 2, 3, 5, p - 1):
        T = oracle_mod.PrefixTable(p, a, stride)
        brute = [0]
        for i in range(1, p):
            brute.append(brute[-1] + pow(a, i, p))
        assert brute[-1] == p * (p - 1) // 2
        for t in range(p):
            assert T.pref(t) == brute[t]


@pytest.mark.parametrize("n,p,e", TINY[:6])
def test_state_at_matches_stepping_tiny(oracle_mod, n, p, e):
    a = primitive_root(p)
    rng = random.Random(n + p)
    T = oracle_mod.PrefixTable(p, a, 3)
    for _ in range(60):
        m0, L0 = rng.randrange(n), rng.randrange(p - 1)
        s0 = pow(a, L0, p)
        t = rng.randrange(0, 4 * n * (p - 1))
        _, _, st = oracle_mod.generate(n, e, p, a, m0, s0, t)
        assert T.state_at(n, m0, L0, t) == st


def test_dlog_places_seeds_on_the_cycle(oracle_mod):
    rng = random.Random(10)
    s = [1, A31, P31 - 1] + [rng.randrange(1, P31) for _ in range(200)]
    L = oracle_mod.dlog(P31, A31, s)
    for si, li in zip(s, L):
        assert 0 <= int(li) < P31 - 1 and pow(A31, int(li), P31) == si


@pytest.mark.slow
def test_default_skip_cycle_sum_and_state_at(oracle_mod):
    """Full cycle of (p, a) = (2^31-1, 784588716): Pref(p-1) = p(p-1)/2, and
    Eq. 7 from a seed agrees with Eq. 7 by stepping at offsets past one cycle."""
    T = oracle_mod.PrefixTable(P31, A31, 1 << 16)
    assert T.pref(P31 - 1) == P31 * (P31 - 1) // 2
    rng = random.Random(11)
    n = 4294967087
    for _ in range(6):
        m0, s0 = rng.randrange(n), rng.randrange(1, P31)
        L0 = int(oracle_mod.dlog(P31, A31, [s0])[0])
        t = rng.randrange(0, 1 << 40)
        k_small = rng.randrange(0, 3000)
        st = T.state_at(n, m0, L0, t)
        # stepping agrees after a further k_small steps
        _, _, st2 = oracle_mod.generate(n, 9, P31, A31, st[0], st[1], k_small)
        assert T.state_at(n, m0, L0, t + k_small) == st2
        # and the q-cycle term matches Eq. 7 by stepping for offsets q(p-1)+r
        r = rng.randrange(0, 5000)
        t2 = (t // (P31 - 1)) * (P31 - 1) + r
        assert T.state_at(n, m0, L0, t2) == oracle_mod.skip_stepping(n, P31, A31, m0, s0, t2)


# ------------------------------------------------------------ fused statistics
@pytest.mark.parametrize("n,p,e", TINY[:6])
def test_stats_full_period_closed_forms(oracle_mod, n, p, e):
    a = primitive_root(p)
    P = n * (p - 1)
    c, _, _ = oracle_mod.generate(n, e, p, a, 3 % n, 1, P)
    X, Y, hist, mean, var = oracle_mod.stats(c, n)
    assert X == (p - 1) * n * (n + 1) // 2
    assert Y == (p - 1) * n * (n + 1) * (2 * n + 1) // 6
    expect = np.zeros(256, dtype=np.int64)
    for cc in range(n):
        expect[(256 * (cc + 1)) // (n + 1)] += p - 1
    assert np.array_equal(hist.astype(np.int64), expect)
    assert mean == float(X) / float(P * (n + 1))
    assert var == float(P * Y - X * X) / float(P * (P - 1) * (n + 1) ** 2)
    # mean of (c+1)/(n+1) over a uniform full period is 1/2 exactly
    assert Fraction(X, P * (n + 1)) == Fraction(1, 2)


def test_corr_pins(oracle_mod):
    rng = random.Random(12)
    n1, n2 = 4294967087, 4294967291
    c1, _, _ = oracle_mod.generate(n1, 9, P31, A31, rng.randrange(n1), 5, 3000)
    c2, _, _ = oracle_mod.generate(n2, 17, P31, A31, rng.randrange(n2), 7, 3000)
    X1, Y1, *_ = oracle_mod.stats(c1, n1)
    X2, Y2, *_ = oracle_mod.stats(c2, n2)
    Z11, _ = oracle_mod.corr(c1, c1, n1, n1)
    assert Z11 == Y1                                  # identical streams
    Z12, corr = oracle_mod.corr(c1, c2, n1, n2)
    assert Z12 * Z12 <= Y1 * Y2                       # Cauchy-Schwarz
    assert corr == float(Z12) / float(3000 * (n1 + 1) * (n2 + 1))
    assert abs(corr - 0.25) < 0.02                    # independent uniforms


def test_u128_conversion_in_stats_is_correctly_rounded(oracle_mod):
    """Large accumulators: mean and var use RN conversions of 128-bit integers."""
    n = 4294967291
    rng = random.Random(13)
    c = np.array([rng.randrange(n) for _ in range(4097)], dtype=np.uint64)
    X, Y, _, mean, var = oracle_mod.stats(c, n)
    N = c.size
    assert X == sum(int(x) + 1 for x in c)
    assert Y == sum((int(x) + 1) ** 2 for x in c)
    assert bits(mean) == bits(float(X) / float(N * (n + 1)))
    assert bits(var) == bits(float(N * Y - X * X) / float(N * (N - 1) * (n + 1) ** 2))


def test_generate_many_matches_generate(oracle_mod):
    from paper_1411_2484_gb300 import workloads
    inst = workloads.draw_instances(7, seed=99)
    rows = workloads.instance_rows(inst)
    c, r, st, _ = oracle_mod.generate_many(rows, 333, threads=3)
    for i in range(7):
        n, e, p, a, m, s = (int(x) for x in rows[i])
        ci, ri, sti = oracle_mod.generate(n, e, p, a, m, s, 333)
        assert np.array_equal(c[i], ci) and np.array_equal(r[i].view(np.uint64), ri.view(np.uint64))
        assert tuple(int(x) for x in st[i]) == sti


# ------------------------------------------------------------ serial tests
def double_bin(c, n, B):
    """floor(B R) on the double: R = (c+1)/(n+1) correctly rounded (Python's
    true division of integers), then one IEEE double product by B, truncated."""
    return int(((c + 1) / (n + 1)) * B)


def low_exact_multiples(B):
    """k in 1..B-1 whose double product RN(RN(k/B) B) falls below k."""
    return [k for k in range(1, B) if (k / B) * B < k]


@pytest.mark.parametrize("n,p,e", TINY[:6])
@pytest.mark.parametrize("B", [3, 8, 100])
def test_serial_1d_full_period(oracle_mod, n, p, e, B):
    """One-dimensional frequency test over a full period: every c appears
    p-1 times, so bin b holds p-1 times the count of c with floor(B R) = b; for
    these moduli no (c+1)/(n+1) is an exact k/B below its double product, so
    the bins are also the exact rationals floor(B (c+1)/(n+1))."""
    a = primitive_root(p)
    P = n * (p - 1)
    c, _, _ = oracle_mod.generate(n, e, p, a, 2 % n, 1, P)
    hist = oracle_mod.serial_hist(c, n, 1, B)
    expect = np.zeros(B, dtype=np.int64)
    for cc in range(n):
        assert double_bin(cc, n, B) == (B * (cc + 1)) // (n + 1)
        expect[(B * (cc + 1)) // (n + 1)] += p - 1
    assert np.array_equal(hist.astype(np.int64), expect)


def test_exact_multiples_whose_double_product_falls_below():
    """The double product RN(RN(k/B) B) is below k only at a few exact
    multiples: none for B = 10, 1000 and 3 2^j, k = 29, 57, 58 for the paper's
    three-dimensional B = 100 (RN(0.29) 100 = 28.999999999999996)."""
    assert low_exact_multiples(100) == [29, 57, 58]
    assert (29 / 100) * 100 == 28.999999999999996
    for B in [10, 1000] + [3 << j for j in range(11)] + [1 << j for j in range(21)]:
        assert low_exact_multiples(B) == [], B


# n = 2147483999 is prime with n + 1 = 100 * 21474840, so (c+1)/(n+1) = k/100
# exactly for c = 21474840 k - 1.
N100 = 2147483999
B100_CASES = [(622770359, 28), (1224065879, 56), (1245540719, 57)]   # k = 29, 57, 58


def _prime_with_divisor(B, start):
    """The first prime n >= start with B dividing n + 1 (Python Rabin-Miller by pow)."""
    def is_prime(q):
        if q < 2 or any(q % d == 0 for d in (2, 3, 5, 7, 11, 13)):
            return q in (2, 3, 5, 7, 11, 13)
        d, r = q - 1, 0
        while d % 2 == 0:
            d //= 2
            r += 1
        for b in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            x = pow(b, d, q)
            if x in (1, q - 1):
                continue
            for _ in range(r - 1):
                x = x * x % q
                if x == q - 1:
                    break
            else:
                return False
        return True
    n = start + (-1 - start) % B
    while not is_prime(n):
        n += B
    return n


@pytest.mark.parametrize("B", [10, 100, 1000, 3 << 5, 3 << 10])
def test_serial_bins_at_exact_multiples_follow_the_double(oracle_mod, B):
    """Every exact multiple k/B of a prime with B | n + 1, and the number just
    below it: bin k, except k - 1 where the double product falls below k."""
    assert N100 == _prime_with_divisor(100, N100)
    n = N100 if B == 100 else _prime_with_divisor(B, 3_000_000_000)
    low = set(low_exact_multiples(B))
    t = (n + 1) // B
    ks = range(1, B) if B <= 1000 else list(range(1, 40)) + list(range(B - 40, B))
    cs, want = [], []
    for k in ks:
        cs += [k * t - 1, k * t - 2]
        want += [k - 1 if k in low else k, k - 1]
    for c, b in zip(cs, want):
        assert double_bin(c, n, B) == b
    h = oracle_mod.serial_hist(np.array(cs, dtype=np.uint64), n, 1, B)
    expect = np.bincount(np.array(want), minlength=B).astype(np.uint64)
    assert np.array_equal(h, expect)


def test_double_bin_cases_of_the_three_dimensional_serial_test(oracle_mod):
    """The paper's D = 3, B = 100 serial test on n = 2147483999: the three
    exact multiples with a low double product each fall one bin below the
    exact quotient, in the serial, interstream and collision binnings."""
    for c, b in B100_CASES:
        assert (100 * (c + 1)) % (N100 + 1) == 0 and 100 * (c + 1) // (N100 + 1) == b + 1
        assert double_bin(c, N100, 100) == b
        h = oracle_mod.serial_hist(np.array([c], dtype=np.uint64), N100, 1, 100)
        assert int(h[b]) == 1
        # a triple: (c, c, 0) -> b + 100 b + 0
        h3 = oracle_mod.serial_hist(np.array([c, c, 0], dtype=np.uint64), N100, 3, 100)
        assert int(h3[b + 100 * b]) == 1
        hi = oracle_mod.interstream_serial_hist(np.array([[c, 5], [7, c]], dtype=np.uint64),
                                                np.array([N100, N100], dtype=np.uint64), 1, 100)
        assert int(hi[b]) == 2
        # collision: c shares its double bin with a number of exact bin b
        other = b * ((N100 + 1) // 100) + 12345
        assert (100 * (other + 1)) // (N100 + 1) == b
        hc = oracle_mod.collision_hist(np.array([other, c], dtype=np.uint64), N100, 2, 100, 3)
        assert list(hc) == [0, 1, 0]


@pytest.mark.parametrize("D,B", [(1, 1 << 20), (2, 1 << 10), (3, 100), (4, 32), (5, 16)])
def test_serial_tuple_count_and_marginals(oracle_mod, D, B):
    """The paper's bin counts per dimension: floor(N/D) tuples, and the
    marginal of each coordinate equals the one-dimensional histogram of that
    coordinate's numbers (every D-th number)."""
    rng = random.Random(D * 7)
    n = 4294967087
    N = 5000 + rng.randrange(D)
    c, _, _ = oracle_mod.generate(n, 9, P31, A31, rng.randrange(n), 5, N)
    hist = oracle_mod.serial_hist(c, n, D, B)
    ntup = N // D
    assert int(hist.sum()) == ntup
    shaped = hist.reshape((B,) * D)        # index b_0 + B b_1 + ...: axis D-1-d is coordinate d
    for d in range(D):
        axes = tuple(x for x in range(D) if x != D - 1 - d)
        marg = shaped.sum(axis=axes)
        ref = np.zeros(B, dtype=np.uint64)
        for k in range(ntup):
            ref[(B * (int(c[k * D + d]) + 1)) // (n + 1)] += 1
        assert np.array_equal(marg, ref), d
    # accumulation: a second stream adds to the same histogram
    hist2 = oracle_mod.serial_hist(c, n, D, B, hist.copy())
    assert np.array_equal(hist2, 2 * hist)


def test_serial_bin_edges_exact_multiples(oracle_mod):
    """(c+1)/(n+1) exactly k/B falls in bin k; just below it in bin k-1."""
    n = 255 * 4096 + 4095                        # n + 1 = 2^20
    for B in (2, 16, 1 << 10):
        for k in (1, B // 2, B - 1):
            v = k * ((n + 1) // B)
            h = oracle_mod.serial_hist(np.array([v - 1, v - 2], dtype=np.uint64), n, 1, B)
            assert h[k] == 1 and h[k - 1] == 1


# ------------------------------------------------------------ interstream serial test
def test_interstream_one_stream_is_the_serial_test(oracle_mod):
    """With Np = 1 the interleaved order is the stream itself."""
    n = 4294967087
    c, _, _ = oracle_mod.generate(n, 9, P31, A31, 12345, 77, 3001)
    for D, B in ((1, 64), (2, 32), (3, 10), (5, 4)):
        a = oracle_mod.serial_hist(c, n, D, B)
        b = oracle_mod.interstream_serial_hist(c.reshape(1, -1), [n], D, B)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("Np,L,D,B", [(2, 7, 2, 4), (3, 5, 2, 3), (5, 8, 3, 4), (7, 9, 4, 2), (4, 6, 1, 8)])
def test_interstream_against_the_order_built_by_hand(oracle_mod, Np, L, D, B):
    """The paper's order R_1 of streams 0 .. Np-1, then R_2 of each, and so
    on, built with Python loops; bins floor(B R) from correctly rounded
    Python divisions; tuples of D consecutive entries, the tail left out."""
    rng = random.Random(Np * 100 + L)
    ns = [4294967087, 4294967291, 2147483659, 3221225473, 4294967029, 2147483693, 3000000019][:Np]
    c = np.zeros((Np, L), dtype=np.uint64)
    for a in range(Np):
        c[a], _, _ = oracle_mod.generate(ns[a], 9, P31, A31, rng.randrange(ns[a]), 1 + a, L)
    seq = []
    for j in range(L):
        for a in range(Np):
            seq.append(int(B * ((int(c[a, j]) + 1) / (ns[a] + 1))))
    want = np.zeros(B ** D, dtype=np.uint64)
    for t in range(len(seq) // D):
        want[sum(seq[t * D + d] * B ** d for d in range(D))] += 1
    got = oracle_mod.interstream_serial_hist(c, ns, D, B)
    assert np.array_equal(got, want)


def test_interstream_1d_is_the_sum_of_the_streams(oracle_mod):
    """Interleaving does not change a one-dimensional histogram."""
    ns = [4294967087, 4294967291, 2147483659]
    c = np.stack([oracle_mod.generate(n, 17, P31, A31, 99 + k, 3 + k, 2000)[0] for k, n in enumerate(ns)])
    h = oracle_mod.interstream_serial_hist(c, ns, 1, 1 << 10)
    ref = np.zeros(1 << 10, dtype=np.uint64)
    for k, n in enumerate(ns):
        oracle_mod.serial_hist(c[k], n, 1, 1 << 10, ref)
    assert np.array_equal(h, ref)


# ------------------------------------------------------------ poker test
def test_poker_hands_from_chosen_denominations(oracle_mod):
    """n + 1 = 10 t makes floor(10 (c+1)/(n+1)) = d for c = d t (d < 10):
    hands of chosen denominations fall in their categories."""
    t = 429496729
    n = 10 * t - 1
    hands = {0: [0, 1, 2, 3, 4], 1: [7, 7, 1, 2, 3], 2: [5, 5, 9, 9, 0], 3: [4, 4, 4, 8, 1],
             4: [2, 2, 2, 6, 6], 5: [3, 3, 3, 3, 9], 6: [8, 8, 8, 8, 8]}
    cs = []
    for cat in range(7):
        cs += [d * t for d in hands[cat]]
    cs += [5 * t, 6 * t]                                   # a remainder of two is left out
    h = oracle_mod.poker_hist(np.array(cs, dtype=np.uint64), n)
    assert list(h) == [1] * 7
    # a permuted hand is the same category; accumulation adds
    h2 = oracle_mod.poker_hist(np.array([d * t for d in [6, 2, 6, 2, 2]], dtype=np.uint64), n, h.copy())
    assert list(h2 - h) == [0, 0, 0, 0, 1, 0, 0]


def test_poker_frequencies_of_a_long_stream(oracle_mod):
    """Category frequencies of 400,000 hands against the exact probabilities
    (each within 5 standard deviations)."""
    n = 4294967087
    c, _, _ = oracle_mod.generate(n, 9, P31, A31, 12345, 678, 2_000_000)
    h = oracle_mod.poker_hist(c, n).astype(np.float64)
    hands = 400_000
    assert h.sum() == hands
    prob = np.array([0.3024, 0.504, 0.108, 0.072, 0.009, 0.0045, 0.0001])
    z = (h - hands * prob) / np.sqrt(hands * prob * (1 - prob))
    assert np.all(np.abs(z) < 5), z


# ------------------------------------------------------------ runs test
def test_runs_from_chosen_bits(oracle_mod):
    """c below (n-1)/2 gives R <= 1/2 (bit 0), above gives bit 1; c = (n-1)/2
    gives R = 1/2 exactly, bit 0."""
    n = 1000003
    lo, hi, half = 5, n - 7, (n - 1) // 2
    bits = [0, 0, 1, 1, 1, 0, 1, 0, 0, 0, 0, 0, 1, 1]        # runs 2,3,1,1,5 then an open run of 2
    cs = np.array([half if (b == 0 and k == 3 + 2) else (lo if b == 0 else hi)
                   for k, b in enumerate(bits)], dtype=np.uint64)
    h = oracle_mod.runs_hist(cs, n, 4)
    want = np.zeros(8, dtype=np.uint64)
    for b, L in [(0, 2), (1, 3), (0, 1), (1, 1), (0, 5)]:
        want[b * 4 + min(L, 4) - 1] += 1
    assert np.array_equal(h, want)


def test_runs_lengths_of_a_long_stream(oracle_mod):
    """Completed runs cover every number but the open run; run lengths of a
    long stream follow 2^-L (each of the first eight lengths within 5 sigma)."""
    n = 4294967087
    N = 1_000_000
    c, _, _ = oracle_mod.generate(n, 9, P31, A31, 4242, 77, N)
    lmax = 32
    h = oracle_mod.runs_hist(c, n, lmax)
    bits = (c > (n - 1) // 2).astype(np.int64)
    open_run = 1
    while open_run < N and bits[N - 1 - open_run] == bits[N - 1]:
        open_run += 1
    h64 = oracle_mod.runs_hist(c, n, 64)                   # no run reaches 64 here
    lengths = np.concatenate([np.arange(1, 65)] * 2)
    assert h64[63] == 0 and h64[127] == 0
    assert int((h64.astype(np.int64) * lengths).sum()) == N - open_run
    runs = h.astype(np.float64).reshape(2, lmax).sum(axis=0)
    total = runs.sum()
    for L in range(1, 9):
        p = 0.5 ** L
        z = (runs[L - 1] - total * p) / np.sqrt(total * p * (1 - p))
        assert abs(z) < 5, (L, z)


# ------------------------------------------------------------ full-period pattern
@pytest.mark.parametrize("n,p,e", [(23, 11, 3), (107, 53, 5), (1019, 509, 3), (1031, 103, 7)])
@pytest.mark.parametrize("D,nb,c_lo,L0", [(2, 8, 0, None), (3, 5, 2, 9), (4, 3, 0, 40)])
def test_pattern_equals_full_period_brute_force(oracle_mod, n, p, e, D, nb, c_lo, L0):
    """The O(p L0) enumeration equals counting, over a whole period n(p-1) of
    the generator, the D-tuples whose first number lies in [c_lo, c_lo+L0)."""
    if L0 is None:
        L0 = n - c_lo
    L0 = min(L0, n - c_lo)
    a = primitive_root(p)
    P = n * (p - 1)
    c, _, _ = oracle_mod.generate(n, e, p, a, 4 % n, 3 % p or 1, P)
    L1 = -(-n // nb)
    want = np.zeros(nb ** (D - 1), dtype=np.uint64)
    for k in range(P):
        if c_lo <= c[k] < c_lo + L0:
            idx = 0
            for j in range(1, D):
                idx += (int(c[(k + j) % P]) // L1) * nb ** (j - 1)
            want[idx] += 1
    got = oracle_mod.pattern_hist(n, e, p, a, c_lo, L0, D, nb)
    assert np.array_equal(got, want)


def test_pattern_2d_whole_range_is_uniform(oracle_mod):
    """D = 2 over every c0: each value c1 appears p-1 times."""
    n, p, e = 1019, 509, 3
    a = primitive_root(p)
    nb = 7
    got = oracle_mod.pattern_hist(n, e, p, a, 0, n, 2, nb)
    L1 = -(-n // nb)
    want = np.array([(p - 1) * len(range(b * L1, min((b + 1) * L1, n))) for b in range(nb)],
                    dtype=np.uint64)
    assert np.array_equal(got, want)


# ------------------------------------------------------------ collision test
def test_collisions_from_chosen_bins(oracle_mod):
    """n + 1 = 16 t makes floor(16 (c+1)/(n+1)) = b for c = b t: segments of
    eight numbers into 16 bins with known collision counts."""
    t = 268435453
    n = 16 * t - 1
    segs = [[0, 1, 2, 3, 4, 5, 6, 7],                   # 0 collisions
            [3, 3, 3, 9, 9, 1, 2, 15],                  # 3
            [5, 5, 5, 5, 5, 5, 5, 5]]                   # 7
    cs = np.array([b * t for seg in segs for b in seg] + [1, 2, 3], dtype=np.uint64)   # remainder
    h = oracle_mod.collision_hist(cs, n, 8, 16, 6)
    assert list(h) == [1, 0, 0, 1, 0, 1]                # 7 collisions capped into the last counter


def test_collision_mean_of_a_long_stream(oracle_mod):
    """The paper's sizes (2^14 numbers into 2^20 bins): the mean collision count
    over 120 segments within 5 standard errors of S - B (1 - (1 - 1/B)^S)."""
    n = 4294967087
    S, B, H = 1 << 14, 1 << 20, 512
    c, _, _ = oracle_mod.generate(n, 9, P31, A31, 99, 12345, 120 * S + 17)
    h = oracle_mod.collision_hist(c, n, S, B, H)
    assert int(h.sum()) == 120
    mean = float((h * np.arange(H)).sum()) / 120
    expect = S - B * (1 - (1 - 1 / B) ** S)
    assert abs(mean - expect) < 5 * np.sqrt(expect / 120), (mean, expect)


@pytest.mark.parametrize("n,e", [(23, 3), (1019, 3), (4099, 5)])
@pytest.mark.parametrize("b", [1, 7])
@pytest.mark.parametrize("D,nb,c_lo,L0", [(2, 8, 0, None), (3, 5, 3, 11), (4, 3, 0, 200)])
def test_pattern_const_equals_full_period_brute_force(oracle_mod, n, e, b, D, nb, c_lo, L0):
    """The constant-skip (b = 1: unit skip) pattern equals counting the D-tuples
    of a whole period m_k = m_0 + k b, c_k = m_k^e mod n."""
    L0 = min(n - c_lo if L0 is None else L0, n - c_lo)
    c = [pow((5 + k * b) % n, e, n) for k in range(n)]
    L1 = -(-n // nb)
    want = np.zeros(nb ** (D - 1), dtype=np.uint64)
    for k in range(n):
        if c_lo <= c[k] < c_lo + L0:
            idx = 0
            for j in range(1, D):
                idx += (c[(k + j) % n] // L1) * nb ** (j - 1)
            want[idx] += 1
    got = oracle_mod.pattern_const_hist(n, e, b, c_lo, L0, D, nb)
    assert np.array_equal(got, want)


# ------------------------------------------------------------ Fourier test
def test_fourier_pure_tone_and_parseval(oracle_mod):
    """A pure tone x_j = cos(2 pi j k0 / M) has xhat_k0 = sqrt(M)/2 and no other
    coefficient in 1 .. M/2-1; Parseval: the coefficients of the full circle
    carry sum x_j^2."""
    import oracle as om
    M, k0 = 4096, 37
    j = np.arange(M)
    R = 0.5 + np.cos(2 * np.pi * j * k0 / M)
    X = om.fourier_coefficients(R, M)[0]
    assert abs(X[k0] - np.sqrt(M) / 2) < 1e-9
    others = np.delete(np.abs(X[1:]), k0 - 1)
    assert others.max() < 1e-9
    rng = np.random.default_rng(5)
    R = rng.random(M)
    X = om.fourier_coefficients(R, M)[0]
    full = np.fft.fft(R - 0.5) / np.sqrt(M)              # the whole circle
    assert abs(np.sum(np.abs(full) ** 2) - np.sum((R - 0.5) ** 2)) < 1e-9
    # the kept half equals the conjugate-symmetric half of the full transform
    assert np.allclose(X, np.conj(full[: M // 2]))


def test_fourier_direct_sum_and_bin_edges(oracle_mod):
    """Brute force on a tiny input: the definition summed term by term with
    complex exponentials, for two sequences of M = 64; and bin edges: a part
    exactly at -w + 2w b / nbins falls in bin b."""
    import cmath
    import oracle as om
    M = 64
    rng = np.random.default_rng(11)
    R = rng.random(2 * M)
    X = om.fourier_coefficients(R, M)
    assert X.shape == (2, M // 2)
    for s in range(2):
        for k in range(M // 2):
            want = sum((R[s * M + j] - 0.5) * cmath.exp(2j * cmath.pi * j * k / M)
                       for j in range(M)) / M ** 0.5
            assert abs(X[s, k] - want) < 1e-12
    for nbins, w in ((64, 1.0), (8, 0.5), (4096, 2.0)):
        for b in (0, 1, nbins // 2, nbins - 1):
            assert om.fourier_bin(-w + 2 * w * b / nbins, nbins, w) == b
            assert om.fourier_bin(-w + 2 * w * (b + 1) / nbins - 1e-9, nbins, w) == b


def test_fourier_variance_one_over_24(oracle_mod):
    """Coefficients of the generator's numbers: real and imaginary parts with
    variance 1/24 (within 2 %), mean about zero."""
    import oracle as om
    n = 4294967087
    M = 1 << 16
    c, r, _ = oracle_mod.generate(n, 9, P31, A31, 31337, 4242, 4 * M)
    X = om.fourier_coefficients(r, M)[:, 1:].reshape(-1)
    for part in (X.real, X.imag):
        assert abs(part.var() * 24 - 1) < 0.02
        assert abs(part.mean()) < 0.01
    h = om.fourier_hist(X, 64, 1.0)
    assert int(h.sum()) == 2 * X.size
    assert om.fourier_bin(-1.0, 64, 1.0) == 0 and om.fourier_bin(0.999999, 64, 1.0) == 63
    assert om.fourier_bin(5.0, 64, 1.0) == 63 and om.fourier_bin(-5.0, 64, 1.0) == 0


# ------------------------------------------------------------ pattern regions (Figs. 2-4)
@pytest.mark.parametrize("n,p,e,D,nb", [(23, 11, 3, 2, 4), (47, 23, 5, 3, 3), (1019, 509, 3, 2, 7)])
def test_pattern_region_full_range_reduction(oracle_mod, n, p, e, D, nb):
    """With L1 = ceil(n / nb) the region is the whole range: equal to the
    full-range functions (pseudorandom and unit skip)."""
    a = primitive_root(p)
    L1 = -(-n // nb)
    L0 = min(n, 40)
    assert np.array_equal(oracle_mod.pattern_region_hist(n, e, p, a, 0, L0, D, nb, L1),
                          oracle_mod.pattern_hist(n, e, p, a, 0, L0, D, nb))
    assert np.array_equal(oracle_mod.pattern_const_region_hist(n, e, 1, 0, L0, D, nb, L1),
                          oracle_mod.pattern_const_hist(n, e, 1, 0, L0, D, nb))


@pytest.mark.parametrize("n,p,e,D,nb,L1,c_lo,L0", [(23, 11, 3, 2, 4, 3, 0, 23), (23, 11, 3, 3, 3, 5, 2, 9),
                                                  (47, 23, 5, 2, 5, 4, 10, 20), (47, 23, 5, 3, 2, 9, 0, 47)])
def test_pattern_region_equals_full_period_brute_force(oracle_mod, n, p, e, D, nb, L1, c_lo, L0):
    """Counting, over a whole period n(p-1) of the generator, the D-tuples
    that start in [c_lo, c_lo+L0) with every successor below nb L1, in cells
    of width L1."""
    a = primitive_root(p)
    P = n * (p - 1)
    c, _, _ = oracle_mod.generate(n, e, p, a, 4 % n, 3 % p or 1, P)
    want = np.zeros(nb ** (D - 1), dtype=np.uint64)
    for k in range(P):
        if c_lo <= c[k] < c_lo + L0:
            cells = [int(c[(k + j) % P]) // L1 for j in range(1, D)]
            if all(b < nb for b in cells):
                want[sum(b * nb ** i for i, b in enumerate(cells))] += 1
    assert np.array_equal(oracle_mod.pattern_region_hist(n, e, p, a, c_lo, L0, D, nb, L1), want)
    cu = [pow((5 + k) % n, e, n) for k in range(n)]          # unit skip, period n
    want = np.zeros(nb ** (D - 1), dtype=np.uint64)
    for k in range(n):
        if c_lo <= cu[k] < c_lo + L0:
            cells = [cu[(k + j) % n] // L1 for j in range(1, D)]
            if all(b < nb for b in cells):
                want[sum(b * nb ** i for i, b in enumerate(cells))] += 1
    assert np.array_equal(oracle_mod.pattern_const_region_hist(n, e, 1, c_lo, L0, D, nb, L1), want)


def test_pattern_region_fig2_cribs_and_cell_counts(oracle_mod):
    """Fig. 2 (unit skip, n = 2^32 - 5, e = 9): the printed crib pairs (0, 1),
    (1, 512), (512, 19683), (19683, 262144) are points of the pattern; over the
    magnified square [0, 2^20)^2 cut into 16 cells of (2^18)^2 the total is
    close to 2^40 / n (the caption's 16 +- 4 per cell)."""
    h, rows = read_golden("fig2_unit_skip.txt")
    n, e = int(h["n"]), int(h["e"])
    c = [int(r[1]) for r in rows]                          # c for m = 0, 1, 2, 3, 4
    for c0, c1 in zip(c[:-1], c[1:]):
        got = oracle_mod.pattern_const_region_hist(n, e, 1, c0, 1, 2, 1 << 20, 1)
        assert got[c1] == 1 and int(got.sum()) == 1, (c0, c1)
    cells = np.zeros((4, 4), dtype=np.int64)
    for i in range(4):
        cells[i] = oracle_mod.pattern_const_region_hist(n, e, 1, i << 18, 1 << 18, 2, 4, 1 << 18).astype(np.int64)
    expect = (1 << 40) / n                                # 256 points over the square
    assert abs(cells.sum() - expect) < 6 * expect ** 0.5
    assert cells.min() >= 1 and cells.max() <= 16 + 6 * 4


@pytest.mark.parametrize("n,p,e", [(23, 11, 3), (47, 23, 5), (107, 53, 3)])
def test_pattern_region_fig3_each_pair_once_none_on_diagonal(oracle_mod, n, p, e):
    """Fig. 3's properties of the two-dimensional full-period pattern with
    cells of width 1: every (c_k, c_(k+1)) pair occurs at most once, and none
    lies on the diagonal (0 < s < p <= n - 1)."""
    a = primitive_root(p)
    for c0 in range(n):
        row = oracle_mod.pattern_region_hist(n, e, p, a, c0, 1, 2, n, 1)
        assert row.max() <= 1 and row[c0] == 0
        assert int(row.sum()) == p - 1
