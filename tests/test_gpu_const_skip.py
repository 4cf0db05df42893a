"""GPU tests of the constant-skip generator through the C ABI ("Message
skipping algorithms": Eq. 3 with s_k = b for every k; b = 1 is the unit skip,
the cipher in counter mode).  A context selects it with a = 1 (p = 2, s0 = 1
for the unit skip).  Generation, split launches, skip and seek in both
directions, checkpoint/restore and batched requests with offsets are compared
with the oracle's own Eq. 9 stepping, and the Eq. 4 identity
(k b)^e = b^e k^e mod n is checked on the generator's outputs."""
import os

import numpy as np
import pytest

import oracle
from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def const_rows(count, width, p, seed, b=None):
    """Seeded instances (safe primes, random exponents) with the constant
    skip: a = 1, s0 = b (drawn in [1, p-1] when b is None)."""
    inst = workloads.draw_instances(count, width=width, seed=seed)
    rows = workloads.instance_rows(inst).copy()
    rng = np.random.default_rng(seed)
    rows[:, 2] = p
    rows[:, 3] = 1
    rows[:, 5] = b if b is not None else rng.integers(1, p, count)
    return rows


def generate(ph, torch, ctx, first, num, per, wide):
    c = torch.empty(num * per, dtype=torch.int64 if wide else torch.int32, device="cuda")
    r = torch.empty(num * per, dtype=torch.float64, device="cuda")
    ph.phprng_generate(ctx, first, num, per, c, r, None)
    torch.cuda.synchronize()
    cv = c.cpu().numpy().view(np.uint64 if wide else np.uint32).astype(np.uint64)
    return cv.reshape(num, per), r.cpu().numpy().reshape(num, per)


def check_against_oracle(c, r, rows, per):
    oc, orr, ost, _ = oracle.generate_many(rows, per, threads=THREADS)
    assert np.array_equal(c, oc)
    assert np.array_equal(r.view(np.uint64), orr.view(np.uint64))
    return ost


@pytest.mark.parametrize("width", [32, 64])
@pytest.mark.parametrize("p", [2, 65537])
def test_constant_skip_streams_match_oracle(ph, torch, width, p):
    """Three consecutive calls of ragged lengths over 37 streams, and a split
    launch (4 streams x 2^18 numbers, cut into chunks): c exact, R at 0 ULP,
    states continued."""
    rows = const_rows(37, width, p, seed=700 + p + width, b=1 if p == 2 else None)
    ctx = ph.phprng_create(width, rows, 0)
    try:
        cur = rows.copy()
        for per in (1, 777, 4099):
            c, r = generate(ph, torch, ctx, 0, 37, per, width == 64)
            st = check_against_oracle(c, r, cur, per)
            cur[:, 4:6] = st[:, :2]
        for i in (0, 20, 36):
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["pos"]) == (int(cur[i, 4]), int(cur[i, 5]), 1 + 777 + 4099)
    finally:
        ph.phprng_destroy(ctx)
    rows4 = rows[:4]
    ctx = ph.phprng_create(width, rows4, 0)
    try:
        c, r = generate(ph, torch, ctx, 0, 4, 1 << 18, width == 64)
        check_against_oracle(c, r, rows4, 1 << 18)
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("width", [32, 64])
def test_constant_skip_skip_and_seek_match_oracle(ph, torch, width):
    """Skips forward (the closed form m + k b) and seeks back to earlier
    positions give the same numbers as the oracle stepping Eq. 9 through
    every position; a skip of 2^40 + 5 equals two skips of 2^39 + 2 and 3
    and the definition m0 + k b of the message."""
    rows = const_rows(9, width, 65537, seed=741 + width)
    ctx = ph.phprng_create(width, rows, 0)
    try:
        ks = [0, 1, 2, 255, 256, 1000, 65536 + 7, 200003, 3]
        ph.phprng_skip(ctx, list(range(9)), ks)
        cur = rows.copy()
        for i, k in enumerate(ks):
            # the state after k numbers: the oracle's Eq. 9 applied k times
            n, e, p, a, m, s = (int(x) for x in rows[i])
            _, _, st = oracle.generate(n, e, p, a, m, s, k)
            cur[i, 4], cur[i, 5] = st[0], st[1]
        c, r = generate(ph, torch, ctx, 0, 9, 600, width == 64)
        check_against_oracle(c, r, cur, 600)
        # back to position 5 for every stream, then 300 numbers
        ph.phprng_seek(ctx, list(range(9)), [5] * 9)
        back = rows.copy()
        for i in range(9):
            n, e, p, a, m, s = (int(x) for x in rows[i])
            _, _, st = oracle.generate(n, e, p, a, m, s, 5)
            back[i, 4], back[i, 5] = st[0], st[1]
        c, r = generate(ph, torch, ctx, 0, 9, 300, width == 64)
        check_against_oracle(c, r, back, 300)
        # far skips: the definition of the message after k constant skips
        ph.phprng_seek(ctx, [0, 1], [0, 0])
        ph.phprng_skip(ctx, [0, 1, 1], [(1 << 40) + 5, (1 << 39) + 2, (1 << 39) + 3])
        for i in (0, 1):
            s = ph.phprng_get_state(ctx, i)
            n, b, m0 = int(rows[i, 0]), int(rows[i, 5]), int(rows[i, 4])
            assert s["m"] == (m0 + ((1 << 40) + 5) * b) % n and s["s"] == b
            assert s["pos"] == (1 << 40) + 5
    finally:
        ph.phprng_destroy(ctx)


def test_constant_skip_checkpoint_restore(ph, torch):
    """A state saved after some numbers and restored with phprng_set_state
    into a fresh context continues identically, and the redefined seed
    m - pos b comes out as the original m0."""
    rows = const_rows(5, 32, 65537, seed=760)
    ctx = ph.phprng_create(32, rows, 0)
    ctx2 = ph.phprng_create(32, rows, 0)
    try:
        generate(ph, torch, ctx, 0, 5, 1234, False)
        saved = [ph.phprng_get_state(ctx, i) for i in range(5)]
        c1, r1 = generate(ph, torch, ctx, 0, 5, 500, False)
        for i, s in enumerate(saved):
            ph.phprng_set_state(ctx2, i, s["m"], s["s"], s["c"], s["pos"])
        c2, r2 = generate(ph, torch, ctx2, 0, 5, 500, False)
        assert np.array_equal(c1, c2) and np.array_equal(r1.view(np.uint64), r2.view(np.uint64))
        ph.phprng_seek(ctx2, [3], [0])
        c3, _ = generate(ph, torch, ctx2, 3, 1, 10, False)
        oc, _, _ = oracle.generate(*(int(x) for x in rows[3]), 10)
        assert np.array_equal(c3[0], oc)
    finally:
        ph.phprng_destroy(ctx)
        ph.phprng_destroy(ctx2)


def test_constant_skip_batched_offsets_match_oracle(ph, torch):
    """Batched requests at offsets up to 2^40 on a mixed-width constant-skip
    context: each request starts from m0 + offset b (Eq. 3 summed) and equals
    the oracle's Eq. 9 from there."""
    r32 = const_rows(6, 32, 65537, seed=770)
    r64 = const_rows(3, 64, 65537, seed=771)
    rows = np.concatenate([r32, r64])
    ctx = ph.phprng_create(0, rows, 0)
    try:
        rng = np.random.default_rng(772)
        reqs, off = [], 0
        for i, ln in enumerate([1, 300, 4097, 70, 9000, 256, 333, 1025, 5]):
            reqs.append((i, int(rng.integers(0, 1 << 40)), ln, off, off))
            off += ln
        c = torch.zeros(off, dtype=torch.int64, device="cuda")
        r = torch.zeros(off, dtype=torch.float64, device="cuda")
        ph.phprng_generate_batch(ctx, reqs, c, r)
        torch.cuda.synchronize()
        cv, rv = c.cpu().numpy().view(np.uint64), r.cpu().numpy()
        for (i, o, ln, co, _) in reqs:
            n, e, p, a, m0, b = (int(x) for x in rows[i])
            oc, orr, _ = oracle.generate(n, e, p, a, (m0 + o * b) % n, b, ln)
            assert np.array_equal(cv[co:co + ln], oc), i
            assert np.array_equal(rv[co:co + ln].view(np.uint64), orr.view(np.uint64)), i
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("width", [32, 64])
def test_constant_skip_identity_eq4_on_outputs(ph, torch, width):
    """Eq. 4: with m0 = 0 the constant skip b gives c_k = (k b)^e and the unit
    skip c'_k = k^e, so c_k = b^e c'_k mod n for every k -- checked on the
    GPU's own outputs of both streams (same n, e)."""
    base = const_rows(3, width, 2, seed=780 + width, b=1)
    base[:, 4] = 0
    bs = np.array([2, 12345, 65536], dtype=np.uint64)
    withb = base.copy()
    withb[:, 2] = 65537
    withb[:, 5] = bs
    per = 20000
    ctx_u = ph.phprng_create(width, base, 0)
    ctx_b = ph.phprng_create(width, withb, 0)
    try:
        cu, _ = generate(ph, torch, ctx_u, 0, 3, per, width == 64)
        cb, _ = generate(ph, torch, ctx_b, 0, 3, per, width == 64)
        for i in range(3):
            n, e, b = int(base[i, 0]), int(base[i, 1]), int(bs[i])
            be = pow(b, e, n)
            for k in (0, 1, 2, 999, per - 1):
                assert int(cu[i, k]) == pow(k + 1, e, n)
            lhs = [int(x) for x in cb[i]]
            rhs = [be * int(x) % n for x in cu[i]]
            assert lhs == rhs
    finally:
        ph.phprng_destroy(ctx_u)
        ph.phprng_destroy(ctx_b)
