"""GPU tests of wide skip generators through the C ABI: 64-bit moduli with a
skip prime p between 2^32 and 2^63 (the Implementation section's skip
generator for 64-bit n, period n(p-1) up to 2^127).  Generation, skip-ahead
(Eq. 7 with the window sum formed by stepping, whole cycles in closed form)
and seek in both directions are compared with the oracle's Eq. 9 and its own
Eq. 7 by stepping."""
import os

import numpy as np
import pytest

import oracle
from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
# (p, a): a 63-bit safe prime and a 62-bit prime whose p - 1 has a 51-bit prime
# factor (both checked with Pollard's rho in the library and in the CPU
# tests), and the first prime above 2^32
WIDE = [(9223372036854771239, 11), (3094861432531188877, 6), (4294967311, 3)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def wide_rows(count, p, a, seed):
    inst = workloads.draw_instances(count, width=64, seed=seed)
    rows = workloads.instance_rows(inst).copy()
    rng = np.random.default_rng(seed)
    rows[:, 2] = p
    rows[:, 3] = a
    rows[:, 5] = [int(x) for x in rng.integers(1, min(p, 1 << 63) - 1, count, dtype=np.uint64)]
    return rows


def generate(ph, torch, ctx, first, num, per):
    c = torch.empty(num * per, dtype=torch.int64, device="cuda")
    r = torch.empty(num * per, dtype=torch.float64, device="cuda")
    ph.phprng_generate(ctx, first, num, per, c, r, None)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64).reshape(num, per), r.cpu().numpy().reshape(num, per)


def check(c, r, rows, per):
    oc, orr, ost, _ = oracle.generate_many(rows, per, threads=THREADS)
    assert np.array_equal(c, oc)
    assert np.array_equal(r.view(np.uint64), orr.view(np.uint64))
    return ost


@pytest.mark.parametrize("p,a", WIDE)
def test_wide_skip_generation_matches_oracle(ph, torch, p, a):
    """Three consecutive calls of ragged lengths over 21 streams (a few
    instances: the launch is not split), c exact, R = RN(RN(c+1)/RN(n+1)) at
    0 ULP, states continued."""
    rows = wide_rows(21, p, a, seed=800 + a)
    ctx = ph.phprng_create(64, rows, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        cur = rows.copy()
        for per in (1, 515, 3000):
            c, r = generate(ph, torch, ctx, 0, 21, per)
            st = check(c, r, cur, per)
            cur[:, 4:6] = st
        for i in (0, 20):
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["pos"]) == (int(cur[i, 4]), int(cur[i, 5]), 3516)
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("p,a", WIDE)
def test_wide_skip_skip_and_seek_match_oracle(ph, torch, p, a):
    """Skips of up to 3,000,017 steps (and, for the 33-bit p, two whole cycles
    of p - 1 plus 12,345 steps) equal the oracle's Eq. 7 by stepping; seeks back
    to position 9 equal the oracle's stepping from the seed; the numbers that
    follow match."""
    rows = wide_rows(6, p, a, seed=820 + a)
    ctx = ph.phprng_create(64, rows, 0)
    try:
        ks = [1, 2, 1000, 65537, 3_000_017, 2 * (p - 1) + 12345 if p < (1 << 33) else 777]
        ph.phprng_skip(ctx, list(range(6)), ks)
        cur = rows.copy()
        for i, k in enumerate(ks):
            n, e, pp, aa, m, s = (int(x) for x in rows[i])
            cur[i, 4], cur[i, 5] = oracle.skip_stepping(n, pp, aa, m, s, k)
        c, r = generate(ph, torch, ctx, 0, 6, 700)
        check(c, r, cur, 700)
        for i in range(6):
            st = ph.phprng_get_state(ctx, i)
            assert st["pos"] == ks[i] + 700
        ph.phprng_seek(ctx, list(range(6)), [9] * 6)
        back = rows.copy()
        for i in range(6):
            n, e, pp, aa, m, s = (int(x) for x in rows[i])
            back[i, 4], back[i, 5] = oracle.skip_stepping(n, pp, aa, m, s, 9)
        c, r = generate(ph, torch, ctx, 0, 6, 100)
        check(c, r, back, 100)
    finally:
        ph.phprng_destroy(ctx)


def test_wide_skip_checkpoint_and_limits(ph, torch):
    """get_state / set_state carry a stream into a fresh context; batched
    plans and servers, whose tiles start from the prefix table, are refused;
    a skip of more than 2^40 steps beyond whole cycles is refused."""
    p, a = WIDE[0]
    rows = wide_rows(3, p, a, seed=840)
    ctx = ph.phprng_create(64, rows, 0)
    ctx2 = ph.phprng_create(64, rows, 0)
    try:
        generate(ph, torch, ctx, 0, 3, 999)
        saved = [ph.phprng_get_state(ctx, i) for i in range(3)]
        c1, _ = generate(ph, torch, ctx, 0, 3, 300)
        for i, s in enumerate(saved):
            ph.phprng_set_state(ctx2, i, s["m"], s["s"], s["c"], s["pos"])
        c2, _ = generate(ph, torch, ctx2, 0, 3, 300)
        assert np.array_equal(c1, c2)
        with pytest.raises(ph.PhprngError):
            ph.phprng_plan_create(ctx, [(0, 5, 10, 0, 0)])
        with pytest.raises(ph.PhprngError):
            ph.phprng_skip(ctx, [1], [(1 << 40) + 1])
    finally:
        ph.phprng_destroy(ctx)
        ph.phprng_destroy(ctx2)
