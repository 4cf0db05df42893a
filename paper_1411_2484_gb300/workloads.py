"""Seeded synthetic workloads: instance tables and request streams.

This module only draws inputs.  It holds none of the generator's arithmetic
(no skip update, no message update, no exponentiation of messages, no R):
the random numbers the method consumes (primes n, exponents e, seeds m0 and
s0, request lengths, offsets, arrival times) are drawn here and handed, as
plain integers, both to the CUDA library and to the CPU oracle.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented from its
published definition, so draws are identical on every platform and numpy
version.

Draw rules (Beale, arXiv:1411.2484):
  n   prime in [2^31, 2^32) for 32-bit instances, [2^63, 2^64) for 64-bit ones
      (Introduction; Implementation section), safe primes ((n-1)/2 prime) by
      default as the Implementation section recommends, all distinct
      (parameter splitting gives every instance its own modulus);
  e   uniform in [3, n-2] with gcd(e, n-1) = 1 (Eq. 1 and the decryption
      condition, Eq. 2);
  m0  uniform in [0, n);
  s0  uniform in [1, p-1] (the skip generator's state space, Eq. 5);
  (p, a) = (2^31 - 1, 784588716), the skip generator the paper tests with.
"""
import math

import numpy as np

DEFAULT_P = 2147483647
DEFAULT_A = 784588716
M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 stream; ``next()`` returns the next 64-bit output."""

    def __init__(self, seed):
        self.state = int(seed) & M64

    def next(self):
        self.state = (self.state + _GOLDEN) & M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def bulk(self, k):
        """The next k outputs as a numpy uint64 array (same stream)."""
        idx = np.arange(1, k + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(_GOLDEN)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + k * _GOLDEN) & M64
        return z

    def below(self, bound):
        """Uniform integer in [0, bound) (Lemire's multiply-shift; bias < 2^-32)."""
        return (self.next() * int(bound)) >> 64

    def uniform01(self):
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


# ---------------------------------------------------------------- primality
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
_SMALL = [q for q in range(3, 1000) if all(q % d for d in range(2, int(q ** 0.5) + 1))]


def is_prime(n):
    """Deterministic strong-probable-prime test for n < 3.3e24."""
    n = int(n)
    if n < 2:
        return False
    for q in (2,) + tuple(_SMALL[:20]):
        if n % q == 0:
            return n == q
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    # bases 2, 7, 61 decide every n < 4,759,123,141 (Jaeschke 1993); the twelve
    # primes up to 37 decide every n < 3.3e24.
    for g in ((2, 7, 61) if n < 4759123141 else _MR_BASES):
        x = pow(g, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _sieve_ok(cand, safe, limit=600):
    """Boolean mask: candidate (and (cand-1)/2 when safe) has no odd factor < limit."""
    ok = np.ones(cand.shape, dtype=bool)
    small = cand.max(initial=0) < np.uint64(1 << 32)
    c = cand.astype(np.uint32) if small else cand
    half = (c - c.dtype.type(1)) >> c.dtype.type(1)
    for q in _SMALL:
        if q >= limit:
            break
        qq = c.dtype.type(q)
        ok &= (c % qq) != 0
        if safe:
            ok &= (half % qq) != 0
    return ok


def draw_primes(count, lo, hi, rng, safe=True, exclude=()):
    """`count` distinct primes in [lo, hi), safe primes when `safe`."""
    lo, hi = int(lo), int(hi)
    out, seen = [], set(int(x) for x in exclude)
    width = hi - lo
    small_range = width < (1 << 24)
    while len(out) < count:
        if small_range:
            cands = [lo + rng.below(width) for _ in range(4096)]
        else:
            raw = rng.bulk(1 << 18)
            if width == (1 << 31) and lo == (1 << 31):
                cand = (raw >> np.uint64(33)) + np.uint64(1 << 31)
            elif width == (1 << 63) and lo == (1 << 63):
                cand = (raw >> np.uint64(1)) | np.uint64(1 << 63)
            else:
                cand = np.uint64(lo) + raw % np.uint64(width)
            cand = cand | np.uint64(1)
            if safe:   # safe primes above 7 are 11 mod 12
                cand = cand - cand % np.uint64(12) + np.uint64(11)
                cand = cand[(cand >= np.uint64(lo)) & (cand <= np.uint64(hi - 1))]
            cand = cand[_sieve_ok(cand, safe)]
            cands = [int(x) for x in cand]
        for c in cands:
            if c in seen or not (lo <= c < hi):
                continue
            if pow(2, c - 1, c) != 1:
                continue
            if safe and pow(2, (c - 1) // 2 - 1, (c - 1) // 2) != 1:
                continue
            if is_prime(c) and (not safe or is_prime((c - 1) // 2)):
                seen.add(c)
                out.append(c)
                if len(out) == count:
                    break
    return out


def draw_exponent(n, rng, lo=3):
    """e uniform in [lo, n-2] with gcd(e, n-1) = 1."""
    while True:
        e = lo + rng.below(n - 2 - lo + 1)
        if math.gcd(e, n - 1) == 1:
            return e


def draw_instances(count, width=32, seed=0x1411_2484, safe=True, p=DEFAULT_P,
                   a=DEFAULT_A, n_range=None, exponent=None):
    """Instance table {n, e, p, a, m0, s0} as uint64 numpy arrays.

    width 32: n in [2^31, 2^32); width 64: n in [2^63, 2^64); n_range=(lo, hi)
    overrides the range (small moduli for tests).  exponent fixes e for every
    instance (the paper's recommended e = 9 or 17) instead of drawing it."""
    rng = SplitMix64(seed)                       # moduli
    prng = SplitMix64(seed ^ 0x2484141100000001)  # per-instance e, m0, s0 (in order)
    if n_range is None:
        n_range = (1 << 31, 1 << 32) if width == 32 else (1 << 63, 1 << 64)
    lo, hi = n_range
    lo = max(lo, p + 1)
    primes = []
    while len(primes) < count:
        batch = draw_primes(count - len(primes), lo, hi, rng, safe=safe, exclude=primes)
        for n in batch:
            if exponent is not None and math.gcd(exponent, n - 1) != 1:
                continue
            primes.append(n)
    ns, es, m0s, s0s = [], [], [], []
    for n in primes:
        ns.append(n)
        es.append(exponent if exponent is not None else draw_exponent(n, prng))
        m0s.append(prng.below(n))
        s0s.append(1 + prng.below(p - 1))
    u = lambda v: np.array(v, dtype=np.uint64)
    return {"n": u(ns), "e": u(es), "p": u([p] * count), "a": u([a] * count),
            "m0": u(m0s), "s0": u(s0s)}


def instance_rows(inst):
    """uint64[count, 6] rows (n, e, p, a, m0, s0)."""
    return np.stack([inst[k] for k in ("n", "e", "p", "a", "m0", "s0")], axis=1).astype(np.uint64)


def concat_instances(*tables):
    return {k: np.concatenate([t[k] for t in tables]) for k in ("n", "e", "p", "a", "m0", "s0")}


# ------------------------------------------------------------ named workloads
WORKLOADS = {
    # 4 instances x 2^20 numbers, 32-bit safe primes, c and R stored.
    "pr1_ref_32bit_4x2^20": dict(width=32, instances=4, per_inst=1 << 20, calls=1,
                                 seed=0x5EED0000),
    # 65,536 instances x 4,096 numbers per call, 64 calls via stored state.
    "plain32_65536x4096x64": dict(width=32, instances=65536, per_inst=4096, calls=64,
                                  seed=0x5EED0001),
    # The same scale with the paper's small exponent e = 9 for every instance
    # (its recommended setting; 4 products per encryption instead of ~40).
    "plain32_e9_65536x4096": dict(width=32, instances=65536, per_inst=4096, calls=64,
                                  seed=0x5EED0009, exponent=9),
    # 4,096 64-bit safe primes x 2^20 numbers each.
    "wide64_4096x2^20": dict(width=64, instances=4096, per_inst=1 << 20, calls=1,
                             seed=0x5EED0002),
}


def batched_requests(instances32, instances64, max_len=1 << 20, max_offset=1 << 40, seed=7):
    """Requests for the batched workload: one per instance (32-bit instances
    first, then 64-bit), length floor(exp(U ln max_len)) in [1, max_len]
    (log-uniform), start offset uniform in [0, max_offset), outputs packed
    one after another (c and R at the same element offsets)."""
    rng = SplitMix64(seed)
    total = instances32 + instances64
    reqs = np.zeros(total, dtype=[(k, "<u8") for k in ("inst", "offset", "len", "c_off", "r_off")])
    off = 0
    for i in range(total):
        length = int(math.floor(math.exp(rng.uniform01() * math.log(max_len))))
        length = min(max(length, 1), max_len)
        reqs[i] = (i, rng.below(max_offset), length, off, off)
        off += length
    return reqs


WORKLOADS["batched_20000_mixed"] = dict(instances32=16000, instances64=4000, max_len=1 << 20,
                                        max_offset=1 << 40, seed=0x5EED0003)


def workload_instances(name, count=None):
    """Instance table of a named workload (optionally only its first `count`)."""
    w = WORKLOADS[name]
    return draw_instances(count or w["instances"], width=w["width"], seed=w["seed"],
                          exponent=w.get("exponent"))
