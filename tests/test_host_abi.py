"""CPU tests of the C ABI: the library loads and exports every declared
symbol; the host-only entry points (primality, validation, seeding) and the
validation path of phprng_create behave as include/phprng.h states.  No call
here launches GPU work."""
import math
import os
import random
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT, read_golden
from paper_1411_2484_gb300 import workloads

P31, A31 = 2147483647, 784588716


def declared_functions():
    src = open(os.path.join(ROOT, "include", "phprng.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phprng_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol(ph):
    names = declared_functions()
    assert len(names) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", ph.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (phprng_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ph._load()
    for n in names:
        assert hasattr(lib, n)
    # nothing but the C ABI is exported
    assert exported == set(names)


def test_binding_names_match_the_abi(ph):
    for n in declared_functions():
        assert callable(getattr(ph, n)), n


def test_is_prime_matches_a_sieve(ph):
    N = 1 << 18
    s = np.ones(N, bool)
    s[:2] = False
    for q in range(2, int(N ** 0.5) + 1):
        if s[q]:
            s[q * q::q] = False
    lib = ph._load()
    assert all(bool(lib.phprng_is_prime(x)) == bool(s[x]) for x in range(N))


def test_is_prime_random_wide(ph):
    rng = random.Random(1)
    for _ in range(3000):
        n = rng.randrange(1 << 20, 1 << 64) | 1
        assert ph.phprng_is_prime(n) == workloads.is_prime(n)
    for n in (4294967291, 4294967087, 18446744073709551557, 2147483647):
        assert ph.phprng_is_prime(n)


def test_paper_bases_reject_strong_pseudoprimes(ph):
    """Each golden number is a strong pseudoprime to every base but the last of
    the paper's list for its range, so a test that dropped a base would call
    it prime (golden: tests/golden/mr_pseudoprimes.txt)."""
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "mr_pseudoprimes.txt")):
        line = line.split("#", 1)[0].split()
        if line:
            n = int(line[0])
            passes = [int(x) for x in line[1].split("=")[1].split(",")]
            fails = int(line[2].split("=")[1])
            rows.append((n, passes, fails))
    assert len(rows) == 2
    for n, passes, fails in rows:
        assert not ph.phprng_is_prime(n)
        d, r = n - 1, 0
        while d % 2 == 0:
            d //= 2
            r += 1

        def sprp(g):
            x = pow(g, d, n)
            if x in (1, n - 1):
                return True
            for _ in range(r - 1):
                x = x * x % n
                if x == n - 1:
                    return True
            return False
        assert all(sprp(g) for g in passes) and not sprp(fails)


def _one(n=4294967087, e=9, p=P31, a=A31, m0=5, s0=7):
    return [(n, e, p, a, m0, s0)]


@pytest.mark.parametrize("inst,width,flags,status", [
    (_one(n=4294967089), 32, 0, 2),                  # composite n
    (_one(n=4294967291), 32, 1, 2),                  # prime but not safe
    (_one(e=2), 32, 0, 3),                           # gcd(e, n-1) != 1
    (_one(e=1), 32, 0, 3),                           # e < 3
    (_one(e=4294967086), 32, 0, 3),                  # e > n-2
    (_one(p=4294967291), 32, 0, 4),                  # p >= n
    (_one(p=2147483649), 32, 0, 4),                  # p composite
    (_one(a=2), 32, 0, 4),                           # 2 is not a primitive root mod 2^31-1
    (_one(s0=0), 32, 0, 4),                          # s0 outside [1, p-1]
    (_one(s0=P31), 32, 0, 4),
    (_one(m0=4294967087), 32, 0, 1),                 # m0 >= n
    (_one(n=18446744073709551557), 32, 0, 1),        # 64-bit n on the 32-bit path
    (_one() + _one(m0=9), 32, 0, 5),                 # duplicate modulus
    (_one() + [(4294967291, 9, 11, 2, 0, 1)], 0, 0, 4),   # two skip generators in one context
    (_one(), 48, 0, 1),                              # bad width
    (_one(p=2, a=1, s0=2), 32, 0, 4),                # constant skip: s0 >= p
    (_one(p=65535, a=1, s0=3), 32, 0, 4),            # constant skip: p composite
    (_one(p=1, a=1, s0=1), 32, 0, 4),                # constant skip: p < 2
    (_one(n=23, e=3, p=23, a=1, s0=1, m0=0), 32, 0, 4),   # constant skip: p >= n
])
def test_validation_errors(ph, inst, width, flags, status):
    rc, bad, msg = ph.phprng_validate(width, inst, flags)
    assert rc == status, (rc, msg)
    assert msg
    # phprng_create fails the same way before touching any device
    with pytest.raises(ph.PhprngError) as ei:
        ph.phprng_create(width, inst, flags)
    assert ei.value.status == status


def test_validation_accepts_paper_parameters(ph):
    assert ph.phprng_validate(32, _one(), 1)[0] == 0
    assert ph.phprng_validate(32, _one() + _one(m0=9), 2)[0] == 0       # shared n allowed
    assert ph.phprng_validate(64, [(18446744073709551557, 3, P31, A31, 0, 1)], 0)[0] == 0
    assert ph.phprng_validate(0, _one() + [(18446744073709551557, 5, P31, A31, 1, 1)], 0)[0] == 0


def test_validation_accepts_constant_skips(ph):
    """a = 1 selects the constant skip s_k = s0 (Eq. 3 with s_k = b): the unit
    skip with p = 2, s0 = 1 (the paper's Fig. 2 generator) and any b < p."""
    assert ph.phprng_validate(32, _one(p=2, a=1, s0=1), 0)[0] == 0
    assert ph.phprng_validate(32, _one(p=65537, a=1, s0=12345), 1)[0] == 0
    assert ph.phprng_validate(64, [(18446744073709551557, 3, 2, 1, 0, 1)], 0)[0] == 0
    assert ph.phprng_validate(32, _one(p=2, a=1, s0=1) + _one(n=4294967291, p=2, a=1, s0=1), 0)[0] == 0


N64 = 18446744073709551557          # a prime above 2^63


def _pr_factors(x):
    """Distinct prime factors by trial division and Pollard's rho (plain Python)."""
    import math as _m

    def is_p(q):
        if q < 2:
            return False
        for d in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            if q % d == 0:
                return q == d
        d, r = q - 1, 0
        while d % 2 == 0:
            d, r = d // 2, r + 1
        for b in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            y = pow(b, d, q)
            if y in (1, q - 1):
                continue
            for _ in range(r - 1):
                y = y * y % q
                if y == q - 1:
                    break
            else:
                return False
        return True

    def rho(q):
        for c in range(1, 100):
            xx = yy = 2
            g = 1
            while g == 1:
                xx = (xx * xx + c) % q
                yy = (yy * yy + c) % q
                yy = (yy * yy + c) % q
                g = _m.gcd(abs(xx - yy), q)
            if g != q:
                return g
        raise AssertionError("no factor")

    out, stack = set(), [x]
    while stack:
        q = stack.pop()
        if q == 1:
            continue
        for d in range(2, 1000):
            while q % d == 0:
                out.add(d)
                q //= d
        if q == 1:
            continue
        if is_p(q):
            out.add(q)
        else:
            g = rho(q)
            stack += [g, q // g]
    return out


def _is_primitive_root(a, p):
    return all(pow(a, (p - 1) // q, p) != 1 for q in _pr_factors(p - 1))


@pytest.mark.parametrize("p,a", [(9223372036854771239, 11), (3094861432531188877, 6),
                                 (8708977279037121833, 3), (6944567280899478719, 11),
                                 (2606314051492085141, 2), (4294967311, 3)])
def test_validation_of_wide_skip_primes(ph, p, a):
    """Skip primes between 2^32 and 2^63 for 64-bit moduli (the paper's 63-bit
    skip generator): a primitive root is accepted and a quadratic residue (a^2)
    refused -- the library factors p - 1 (Pollard's rho; here p - 1 has prime
    factors up to 2^62) and agrees with plain Python throughout."""
    assert workloads.is_prime(p) and _is_primitive_root(a, p)
    assert ph.phprng_validate(64, [(N64, 3, p, a, 5, 7)], 0)[0] == 0
    assert ph.phprng_validate(0, [(N64, 3, p, a, 5, 7)], 0)[0] == 0
    sq = a * a % p
    assert not _is_primitive_root(sq, p)
    assert ph.phprng_validate(64, [(N64, 3, p, sq, 5, 7)], 0)[0] == 4


def test_validation_refuses_bad_wide_skips(ph):
    p = 9223372036854771239
    composite = p + 2
    assert not workloads.is_prime(composite)
    assert ph.phprng_validate(64, [(N64, 3, composite, 11, 5, 7)], 0)[0] == 4
    big = (1 << 63) + 29                                   # a prime at or above 2^63
    while not workloads.is_prime(big):
        big += 2
    assert ph.phprng_validate(64, [(N64, 3, big, 2, 5, 7)], 0)[0] == 4
    assert ph.phprng_validate(64, [(N64, 3, p, 11, 5, p)], 0)[0] == 4     # s0 = p
    # a 32-bit modulus cannot take a skip prime above 2^32 (p < n)
    assert ph.phprng_validate(32, [(4294967087, 9, 4294967311, 3, 5, 7)], 0)[0] == 4


def test_validation_reports_first_bad_index(ph):
    inst = workloads.instance_rows(workloads.draw_instances(50, seed=11)).tolist()
    inst[37] = list(inst[37])
    inst[37][1] = 2                                   # even exponent
    rc, bad, msg = ph.phprng_validate(32, inst, 1)
    assert rc == 3 and bad == 37 and "instance 37" in msg


@pytest.mark.parametrize("width", [32, 64])
def test_draw_instances_follow_the_paper_conditions(ph, width):
    t = ph.phprng_draw_instances(width, 300, seed=1234, flags=1)
    lo, hi = (1 << 31, 1 << 32) if width == 32 else (1 << 63, 1 << 64)
    ns = [int(x) for x in t["n"]]
    assert len(set(ns)) == 300
    for i in range(300):
        n, e, p, a, m0, s0 = (int(t[k][i]) for k in ("n", "e", "p", "a", "m0", "s0"))
        assert lo <= n < hi and workloads.is_prime(n) and workloads.is_prime((n - 1) // 2)
        assert 3 <= e <= n - 2 and math.gcd(e, n - 1) == 1
        assert (p, a) == (P31, A31) and 0 <= m0 < n and 1 <= s0 < p
    assert ph.phprng_validate(width, t, 1)[0] == 0
    t2 = ph.phprng_draw_instances(width, 300, seed=1234, flags=1)
    assert all(np.array_equal(t[k], t2[k]) for k in t)              # deterministic
    t3 = ph.phprng_draw_instances(width, 300, seed=1235, flags=1)
    assert not np.array_equal(t["n"], t3["n"])


def test_draw_instances_prefix_stable(ph):
    a = ph.phprng_draw_instances(32, 50, seed=99)
    b = ph.phprng_draw_instances(32, 20, seed=99)
    assert all(np.array_equal(a[k][:20], b[k]) for k in a)


def test_status_strings(ph):
    for s in range(10):
        assert ph.phprng_status_string(s)


def test_every_entry_point_rejects_null_handles(ph):
    """Each call that takes a context, plan, server or output pointer returns
    PHPRNG_EINVAL when they are NULL (the destroy calls accept NULL and return
    PHPRNG_OK), without touching a GPU: the checks come before any CUDA call."""
    import ctypes
    lib = ph._load()
    host_only = {"phprng_status_string", "phprng_last_error", "phprng_clock_ns", "phprng_is_prime",
                 "phprng_validate", "phprng_draw_instances"}
    for name in ph.EXPORTED:
        if name in host_only:
            continue
        fn = getattr(lib, name)
        args = []
        for t in fn.argtypes or []:
            if t in (ctypes.c_double, ctypes.c_float):
                args.append(1.0)
            elif t in (ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int):
                args.append(0)
            else:
                args.append(None)
        want = ph.PHPRNG_OK if name.endswith("_destroy") else ph.PHPRNG_EINVAL
        assert fn(*args) == want, name
