"""GPU tests of the Eq. 7 skip-ahead through the C ABI.

The device builds its own prefix table of the skip cycle; the oracle checks
it with a different table (stride 2^16, plain loop) and with plain stepping.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu

P31, A31 = 2147483647, 784588716
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def table31():
    return oracle.PrefixTable(P31, A31, 1 << 16)


def gen(ph, torch, ctx, width, first, num, per):
    cdt = torch.int32 if width == 32 else torch.int64
    c = torch.empty(num * per, dtype=cdt, device="cuda")
    r = torch.empty(num * per, dtype=torch.float64, device="cuda")
    ph.phprng_generate(ctx, first, num, per, c, r)
    torch.cuda.synchronize()
    cn = c.cpu().numpy().view(np.uint32 if width == 32 else np.uint64).astype(np.uint64)
    return cn.reshape(num, per), r.cpu().numpy().reshape(num, per)


def test_skip_small_offsets_against_stepping(ph, torch):
    inst = workloads.draw_instances(12, seed=41)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        ks = [0, 1, 2, 31, 32, 1023, 1024, 1025, 4095, 70000, 123457, 999999]
        ph.phprng_skip(ctx, list(range(12)), ks)
        for i, k in enumerate(ks):
            n, e, p, a, m0, s0 = (int(inst[x][i]) for x in ("n", "e", "p", "a", "m0", "s0"))
            _, _, st = oracle.generate(n, e, p, a, m0, s0, k)
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["pos"]) == (st[0], st[1], k), i
        # outputs after the skip continue the stream
        c, r = gen(ph, torch, ctx, 32, 0, 12, 300)
        for i, k in enumerate(ks):
            n, e, p, a, m0, s0 = (int(inst[x][i]) for x in ("n", "e", "p", "a", "m0", "s0"))
            cr, rr, _ = oracle.generate(n, e, p, a, m0, s0, k + 300)
            assert np.array_equal(c[i], cr[k:]) and np.array_equal(r[i].view(np.uint64),
                                                                    rr[k:].view(np.uint64))
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("width", [32, 64])
def test_skip_large_offsets_against_oracle_table(ph, torch, table31, width):
    inst = workloads.draw_instances(40, width=width, seed=42 + width)
    ctx = ph.phprng_create(width, inst, 0)
    try:
        rng = np.random.default_rng(width)
        ks = [int(x) for x in rng.integers(0, 1 << 40, 40)]
        ks[0], ks[1] = (P31 - 1) * 7, (P31 - 1) * 3 + 5           # exact cycles, cycle + 5
        ph.phprng_skip(ctx, list(range(40)), ks)
        L0 = oracle.dlog(P31, A31, inst["s0"])
        c, r = gen(ph, torch, ctx, width, 0, 40, 257)
        for i, k in enumerate(ks):
            n, e = int(inst["n"][i]), int(inst["e"][i])
            m_k, s_k = table31.state_at(n, int(inst["m0"][i]), int(L0[i]), k)
            s = ph.phprng_get_state(ctx, i)
            assert s["pos"] == k + 257
            cr, rr, st = oracle.generate(n, e, P31, A31, m_k, s_k, 257)
            assert np.array_equal(c[i], cr), i
            assert np.array_equal(r[i].view(np.uint64), rr.view(np.uint64)), i
            assert (s["m"], s["s"]) == st
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("n,p", [(23, 11), (1019, 509), (4294967087, 13)])
def test_skip_tiny_cycles(ph, torch, n, p):
    """Skips spanning many cycles of a tiny skip generator (q large, r small)."""
    from test_gpu_parity import primitive_root
    a = primitive_root(p)
    rng = np.random.default_rng(n)
    count = 6
    inst = {"n": [n] * count, "e": [3 if (n - 1) % 3 else 5] * count, "p": [p] * count,
            "a": [a] * count, "m0": [int(x) for x in rng.integers(0, n, count)],
            "s0": [int(x) for x in rng.integers(1, p, count)]}
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_ALLOW_SHARED_N)
    try:
        ks = [0, 1, p - 1, 5 * (p - 1) + 3, int(rng.integers(0, 1 << 40)),
              int(rng.integers(0, 1 << 62))]
        ph.phprng_skip(ctx, list(range(count)), ks)
        for i, k in enumerate(ks):
            st = oracle.skip_stepping(n, p, a, inst["m0"][i], inst["s0"][i], k)
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["pos"]) == (st[0], st[1], k), (i, k)
    finally:
        ph.phprng_destroy(ctx)


def test_repeated_instances_add_and_match_generation(ph, torch):
    inst = workloads.draw_instances(4, seed=44)
    a = ph.phprng_create(32, inst, 0)
    b = ph.phprng_create(32, inst, 0)
    try:
        ph.phprng_skip(a, [2, 0, 2, 2], [1000, 5, 24, 3000])      # instance 2 by 4024
        ph.phprng_skip(a, [1], [0])
        ca, ra = gen(ph, torch, a, 32, 0, 4, 500)
        cb, rb = gen(ph, torch, b, 32, 0, 4, 4024 + 500)
        assert np.array_equal(ca[2], cb[2][4024:])
        assert np.array_equal(ca[0], cb[0][5:505])
        assert np.array_equal(ca[1], cb[1][:500]) and np.array_equal(ca[3], cb[3][:500])
        assert ph.phprng_get_state(a, 2)["pos"] == 4524
        with pytest.raises(ph.PhprngError):
            ph.phprng_skip(a, [4], [1])                              # out of range
        with pytest.raises(ph.PhprngError):
            ph.phprng_skip(a, [0, 0], [2 ** 64 - 1, 2])              # position overflow
    finally:
        ph.phprng_destroy(a)
        ph.phprng_destroy(b)


def test_skip_after_generate_and_c_state(ph, torch):
    """The state's last ciphertext after a skip is Eq. 7c at the new position."""
    inst = workloads.draw_instances(5, seed=45)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        gen(ph, torch, ctx, 32, 0, 5, 77)
        ph.phprng_skip(ctx, list(range(5)), [10 ** 9 + i for i in range(5)])
        for i in range(5):
            s = ph.phprng_get_state(ctx, i)
            assert s["c"] == pow(s["m"], int(inst["e"][i]), int(inst["n"][i]))
            assert s["pos"] == 77 + 10 ** 9 + i
    finally:
        ph.phprng_destroy(ctx)


def test_microbench_rates(ph, torch):
    rates = [ph.phprng_microbench(w) for w in range(12)]
    assert all(r > 1e9 for r in rates), rates
    # the exponent programs run Montgomery products no faster than a bare chain
    assert rates[5] < 1.05 * rates[3], rates
    # R from integers outruns the FP64 division it replaces (GB300's FP64 rate)
    assert rates[7] > rates[6], rates
    print("mul.lo %.3g mad.hi %.3g mad.wide %.3g mont32 %.3g dfma %.3g programs %.3g "
          "div.f64 %.3g R-int %.3g mul.wide %.3g mont32(lo,hi) %.3g mont32c %.3g shoup %.3g per s"
          % tuple(rates))
    with pytest.raises(ph.PhprngError):
        ph.phprng_microbench(12)


@pytest.mark.parametrize("width", [32, 64])
def test_seek_backward_and_forward(ph, torch, table31, width):
    """phprng_seek to absolute positions in both directions (Eq. 7 backward:
    cycle position L - k, message minus the forward window sum): states against
    the oracle's own prefix table, outputs continue the stream, position 0
    restores the seed (c = 0), and a saved position restores the saved state."""
    inst = workloads.draw_instances(8, width=width, seed=46 + width)
    ctx = ph.phprng_create(width, inst, 0)
    try:
        L0 = oracle.dlog(P31, A31, inst["s0"])
        gen(ph, torch, ctx, width, 0, 8, 5000)
        saved = [ph.phprng_get_state(ctx, i) for i in range(8)]
        ph.phprng_skip(ctx, list(range(8)), [(P31 - 1) * 3 + 77] * 8)   # beyond three cycles
        targets = [0, 1, 1234, 4999, 5000, 10 ** 9, (P31 - 1) * 2 + 11, 5000 + (P31 - 1) * 3 + 77]
        ph.phprng_seek(ctx, list(range(8)), targets)
        c, r = gen(ph, torch, ctx, width, 0, 8, 129)
        for i, t in enumerate(targets):
            n, e = int(inst["n"][i]), int(inst["e"][i])
            m_t, s_t = table31.state_at(n, int(inst["m0"][i]), int(L0[i]), t)
            cr, rr, st = oracle.generate(n, e, P31, A31, m_t, s_t, 129)
            assert np.array_equal(c[i], cr), (i, t)
            assert np.array_equal(r[i].view(np.uint64), rr.view(np.uint64)), (i, t)
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["pos"]) == (st[0], st[1], t + 129), (i, t)
        # back to the seed, then to the saved positions
        ph.phprng_seek(ctx, list(range(8)), [0] * 8)
        for i in range(8):
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["c"], s["pos"]) == (int(inst["m0"][i]), int(inst["s0"][i]), 0, 0)
        ph.phprng_seek(ctx, [3, 3, 5], [7, saved[3]["pos"], saved[5]["pos"]])   # last entry wins
        for i in (3, 5):
            s = ph.phprng_get_state(ctx, i)
            assert {k: s[k] for k in ("m", "s", "c", "pos")} == \
                {k: saved[i][k] for k in ("m", "s", "c", "pos")}
        with pytest.raises(ph.PhprngError):
            ph.phprng_seek(ctx, [8], [1])                                # out of range
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("width", [32, 64])
def test_set_state_restores_into_a_fresh_context(ph, torch, table31, width):
    """Checkpoint and restore: states read from one context and written into a
    fresh context of the same instance table continue identically, and the
    restored streams keep their seeds (seeking back to 0 gives m0, s0)."""
    inst = workloads.draw_instances(6, width=width, seed=60 + width)
    a = ph.phprng_create(width, inst, 0)
    b = ph.phprng_create(width, inst, 0)
    try:
        gen(ph, torch, a, width, 0, 6, 3001)
        ph.phprng_skip(a, [2, 4], [10 ** 12, (P31 - 1) * 5 + 3])
        saved = [ph.phprng_get_state(a, i) for i in range(6)]
        for i, st in enumerate(saved):
            ph.phprng_set_state(b, i, st["m"], st["s"], st["c"], st["pos"])
        for i in range(6):
            assert ph.phprng_get_state(b, i) == saved[i]
        ca, ra = gen(ph, torch, a, width, 0, 6, 777)
        cb, rb = gen(ph, torch, b, width, 0, 6, 777)
        assert np.array_equal(ca, cb) and np.array_equal(ra.view(np.uint64), rb.view(np.uint64))
        ph.phprng_seek(b, list(range(6)), [0] * 6)
        for i in range(6):
            s = ph.phprng_get_state(b, i)
            assert (s["m"], s["s"], s["c"], s["pos"]) == (int(inst["m0"][i]), int(inst["s0"][i]), 0, 0)
    finally:
        ph.phprng_destroy(a)
        ph.phprng_destroy(b)


@pytest.mark.parametrize("width", [32, 64])
def test_set_state_arbitrary_against_oracle(ph, torch, table31, width):
    """An arbitrary (m, s) at an arbitrary position: generation continues by
    Eq. 9 from it (oracle), seek forward from it equals stepping the oracle,
    seek back to 0 and forward again returns to it, and a batched request at
    an offset follows the redefined stream."""
    inst = workloads.draw_instances(4, width=width, seed=70 + width)
    ctx = ph.phprng_create(width, inst, 0)
    rng = np.random.default_rng(width)
    try:
        picks = []
        for i in range(4):
            n = int(inst["n"][i])
            m = int(rng.integers(0, n - 1, dtype=np.uint64))
            s = int(rng.integers(1, P31 - 1))
            pos = [0, 17, 10 ** 11 + 5, (P31 - 1) * 7 + 1000][i]
            ph.phprng_set_state(ctx, i, m, s, 12345 % n, pos)
            picks.append((n, int(inst["e"][i]), m, s, pos))
        c, r = gen(ph, torch, ctx, width, 0, 4, 1500)
        for i, (n, e, m, s, pos) in enumerate(picks):
            cr, rr, st = oracle.generate(n, e, P31, A31, m, s, 1500)
            assert np.array_equal(c[i], cr) and np.array_equal(r[i].view(np.uint64), rr.view(np.uint64))
            assert ph.phprng_get_state(ctx, i)["pos"] == pos + 1500
        # forward by seek: 1500 numbers plus 2 full cycles plus 99 beyond the set state
        ph.phprng_seek(ctx, list(range(4)), [p[4] + 1500 + 2 * (P31 - 1) + 99 for p in picks])
        c2, _ = gen(ph, torch, ctx, width, 0, 4, 64)
        for i, (n, e, m, s, pos) in enumerate(picks):
            _, _, st = oracle.generate(n, e, P31, A31, m, s, 1500 + 99)
            # two whole skip cycles add 2 p(p-1)/2 to m and leave s unchanged
            m2 = (int(st[0]) + 2 * (P31 * (P31 - 1) // 2)) % n
            cr, _, _ = oracle.generate(n, e, P31, A31, m2, int(st[1]), 64)
            assert np.array_equal(c2[i], cr), i
        ph.phprng_seek(ctx, list(range(4)), [0] * 4)
        ph.phprng_seek(ctx, list(range(4)), [p[4] for p in picks])
        for i, (n, e, m, s, pos) in enumerate(picks):
            g = ph.phprng_get_state(ctx, i)
            assert (g["m"], g["s"], g["pos"]) == (m, s, pos), i
        # a batched request 250 numbers past the set state
        reqs = np.zeros(1, dtype=[(k, "<u8") for k in ("inst", "offset", "len", "c_off", "r_off")])
        reqs[0] = (1, picks[1][4] + 250, 300, 0, 0)
        rb = torch.empty(300, dtype=torch.float64, device="cuda")
        ph.phprng_generate_batch(ctx, reqs, None, rb)
        torch.cuda.synchronize()
        n, e, m, s, pos = picks[1]
        _, rr, _ = oracle.generate(n, e, P31, A31, m, s, 550)
        assert np.array_equal(rb.cpu().numpy().view(np.uint64), rr[250:].view(np.uint64))
        for bad in ((0, int(inst["n"][0]), 1, 0, 0), (0, 1, 0, 0, 0), (0, 1, P31, 0, 0),
                    (0, 1, 1, int(inst["n"][0]), 0), (4, 1, 1, 0, 0)):
            with pytest.raises(ph.PhprngError):
                ph.phprng_set_state(ctx, *bad)
    finally:
        ph.phprng_destroy(ctx)
