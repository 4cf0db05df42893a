"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

c must match exactly and R bit for bit (0 ULP): for n < 2^32 the correctly
rounded (c+1)/(n+1); for 64-bit n the reading RN(RN(c+1)/RN(n+1)).
Sizes span several warp groups and ragged tails; the plain 32-bit workload
is also checked at full size (65,536 instances x 4,096 numbers per call) in
the launch configuration the benchmark times.
"""
import math
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
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    return t


def generate(ph, torch, ctx, width, first, num, per, want_c=True, want_r=True):
    cdt = torch.int32 if width == 32 else torch.int64
    c = torch.empty(num * per, dtype=cdt, device="cuda") if want_c else None
    r = torch.empty(num * per, dtype=torch.float64, device="cuda") if want_r else None
    ph.phprng_generate(ctx, first, num, per, c, r, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    cn = None
    if want_c:
        cn = c.cpu().numpy().view(np.uint32 if width == 32 else np.uint64).astype(np.uint64)
        cn = cn.reshape(num, per)
    rn = r.cpu().numpy().reshape(num, per) if want_r else None
    return cn, rn


class OracleStreams:
    """Per-instance oracle state, advanced in step with the device."""

    def __init__(self, inst):
        self.rows = workloads.instance_rows(inst).copy()   # n e p a m s (m, s = current)

    def next(self, first, num, per):
        c, r, st, _ = oracle.generate_many(self.rows[first:first + num], per, threads=THREADS)
        self.rows[first:first + num, 4:6] = st
        return c, r


def assert_same(c_gpu, r_gpu, c_ref, r_ref):
    if c_gpu is not None:
        bad = np.argwhere(c_gpu != c_ref)
        assert bad.size == 0, "c differs at %s: gpu %d oracle %d" % (
            tuple(bad[0]), c_gpu[tuple(bad[0])], c_ref[tuple(bad[0])])
    if r_gpu is not None:
        bad = np.argwhere(r_gpu.view(np.uint64) != r_ref.view(np.uint64))
        assert bad.size == 0, "R differs at %s: gpu %r oracle %r" % (
            tuple(bad[0]), r_gpu[tuple(bad[0])], r_ref[tuple(bad[0])])


def check_state(ph, ctx, orc, first, num, pos):
    for i in range(first, first + num):
        s = ph.phprng_get_state(ctx, i)
        assert (s["m"], s["s"], s["pos"]) == (int(orc.rows[i, 4]), int(orc.rows[i, 5]), pos[i])


def test_pr1_ref_4x2p20_full_compare(ph, torch):
    """4 instances x 2^20 numbers, c and R, every element."""
    inst = workloads.workload_instances("pr1_ref_32bit_4x2^20")
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        orc = OracleStreams(inst)
        c, r = generate(ph, torch, ctx, 32, 0, 4, 1 << 20)
        assert_same(c, r, *orc.next(0, 4, 1 << 20))
        check_state(ph, ctx, orc, 0, 4, [1 << 20] * 4)
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("per", [1, 2, 3, 5, 16, 31, 127, 128, 129, 255, 256, 272, 1000, 4097, 4112])
def test_ragged_lengths_and_continuation(ph, torch, per):
    inst = workloads.draw_instances(9, seed=1000 + per)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        orc = OracleStreams(inst)
        for call in range(3):
            c, r = generate(ph, torch, ctx, 32, 0, 9, per)
            assert_same(c, r, *orc.next(0, 9, per))
        check_state(ph, ctx, orc, 0, 9, [3 * per] * 9)
    finally:
        ph.phprng_destroy(ctx)


def test_subranges_c_only_r_only(ph, torch):
    inst = workloads.draw_instances(20, seed=77)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        orc = OracleStreams(inst)
        pos = [0] * 20
        for first, num, per, wc, wr in [(3, 5, 300, True, True), (0, 20, 64, True, False),
                                        (19, 1, 999, False, True), (7, 13, 130, True, True)]:
            c, r = generate(ph, torch, ctx, 32, first, num, per, wc, wr)
            cr, rr = orc.next(first, num, per)
            assert_same(c, r, cr if wc else None, rr if wr else None)
            for i in range(first, first + num):
                pos[i] += per
        check_state(ph, ctx, orc, 0, 20, pos)
    finally:
        ph.phprng_destroy(ctx)


def test_split_calls_equal_one_call_and_alone_equals_batch(ph, torch):
    inst = workloads.draw_instances(16, seed=5)
    a = ph.phprng_create(32, inst, 0)
    b = ph.phprng_create(32, inst, 0)
    try:
        c1, r1 = generate(ph, torch, a, 32, 0, 16, 1000)
        c2, r2 = generate(ph, torch, a, 32, 0, 16, 2333)
        whole_c, whole_r = [], []
        for i in range(16):                               # each instance alone
            c, r = generate(ph, torch, b, 32, i, 1, 3333)
            whole_c.append(c[0])
            whole_r.append(r[0])
        whole_c, whole_r = np.stack(whole_c), np.stack(whole_r)
        assert np.array_equal(np.concatenate([c1, c2], axis=1), whole_c)
        assert np.array_equal(np.concatenate([r1, r2], axis=1).view(np.uint64),
                              whole_r.view(np.uint64))
    finally:
        ph.phprng_destroy(a)
        ph.phprng_destroy(b)


def primitive_root(p):
    fac, x, d = set(), p - 1, 2
    while d * d <= x:
        while x % d == 0:
            fac.add(d)
            x //= d
        d += 1
    if x > 1:
        fac.add(x)
    return next(g for g in range(2, p) if all(pow(g, (p - 1) // q, p) != 1 for q in fac))


@pytest.mark.parametrize("n,p,e", [(23, 11, 3), (107, 53, 5), (1019, 509, 7), (2027, 1013, 3)])
def test_tiny_moduli_full_period(ph, torch, n, p, e):
    """A whole period n(p-1): equal to the oracle, every c exactly p-1 times."""
    a = primitive_root(p)
    inst = {"n": [n], "e": [e], "p": [p], "a": [a], "m0": [3], "s0": [1]}
    ctx = ph.phprng_create(32, inst, 0)
    try:
        P = n * (p - 1)
        c, r = generate(ph, torch, ctx, 32, 0, 1, P)
        orc = OracleStreams({k: np.array(v, dtype=np.uint64) for k, v in inst.items()})
        assert_same(c, r, *orc.next(0, 1, P))
        assert np.all(np.bincount(c[0].astype(np.int64), minlength=n) == p - 1)
        s = ph.phprng_get_state(ctx, 0)
        assert (s["m"], s["s"]) == (3, 1)                 # back to the seed after P
    finally:
        ph.phprng_destroy(ctx)


def test_extreme_parameters(ph, torch):
    """Largest 32-bit prime, p just below n, e at both ends, seeds at the edges."""
    n_max = 4294967291                                    # 2^32 - 5
    p_big = 4294967279                                    # prime, p < n_max
    groups = [
        [(n_max, 3, P31, A31, 0, 1),
         (4294967087, 4294967085, P31, A31, 4294967086, P31 - 1),
         (2147483659, 2147483657, P31, A31, 1, 2)],
        [(n_max, 3, p_big, primitive_root_big(p_big), 123, p_big - 1)],
    ]
    for rows in groups:
        for row in rows:
            assert ph.phprng_validate(32, [row], 0)[0] == 0, row
        inst = {k: np.array([r[j] for r in rows], dtype=np.uint64)
                for j, k in enumerate(("n", "e", "p", "a", "m0", "s0"))}
        ctx = ph.phprng_create(32, inst, 0)
        try:
            orc = OracleStreams(inst)
            for per in (517, 4096):
                c, r = generate(ph, torch, ctx, 32, 0, len(rows), per)
                assert_same(c, r, *orc.next(0, len(rows), per))
                assert np.all(r > 0) and np.all(r < 1)
        finally:
            ph.phprng_destroy(ctx)


def primitive_root_big(p):
    from paper_1411_2484_gb300.workloads import is_prime
    x, fac, d = p - 1, [], 2
    while d * d <= x:
        if x % d == 0:
            fac.append(d)
            while x % d == 0:
                x //= d
        d += 1
    if x > 1:
        fac.append(x)
    assert is_prime(p)
    return next(g for g in range(2, 1000) if all(pow(g, (p - 1) // q, p) != 1 for q in fac))


def test_64bit_small_and_mixed_context(ph, torch):
    i32 = workloads.draw_instances(10, seed=21)
    i64 = workloads.draw_instances(6, width=64, seed=22)
    mixed = workloads.concat_instances(i32, i64)
    ctx64 = ph.phprng_create(64, i64, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    ctxm = ph.phprng_create(0, mixed, 0)
    try:
        orc = OracleStreams(i64)
        for per in (1, 65, 1000, 2048):
            c, r = generate(ph, torch, ctx64, 64, 0, 6, per)
            assert_same(c, r, *orc.next(0, 6, per))
        orm = OracleStreams(mixed)
        for per in (3, 700):
            c, r = generate(ph, torch, ctxm, 0, 0, 16, per)
            assert_same(c, r, *orm.next(0, 16, per))
        check_state(ph, ctxm, orm, 0, 16, [703] * 16)
    finally:
        ph.phprng_destroy(ctx64)
        ph.phprng_destroy(ctxm)


@pytest.mark.parametrize("count,per", [(600, 65536), (2, (1 << 25) + 1000)],
                         ids=["whole_instances", "split_instances"])
def test_host_output_buffers(ph, torch, count, per):
    """Host pointers (pageable numpy, pinned torch) stage through the device:
    several staging blocks of whole instances (> 2^25 numbers), and instances
    longer than one block (each split over blocks)."""
    if True:
        inst = workloads.draw_instances(count, seed=31 + count)
        a = ph.phprng_create(32, inst, 0)
        b = ph.phprng_create(32, inst, 0)
        try:
            c_h = np.empty(count * per, dtype=np.uint32)
            r_h = torch.empty(count * per, dtype=torch.float64, pin_memory=True)
            ph.phprng_generate(a, 0, count, per, c_h, r_h, None)
            c_d, r_d = generate(ph, torch, b, 32, 0, count, per)
            assert np.array_equal(c_h.reshape(count, per).astype(np.uint64), c_d)
            assert np.array_equal(r_h.numpy().reshape(count, per).view(np.uint64),
                                  r_d.view(np.uint64))
            orc = OracleStreams(inst)
            k = min(count, 4)
            cr, rr = orc.next(0, k, min(per, 70000))
            assert_same(c_d[:k, :cr.shape[1]], r_d[:k, :cr.shape[1]], cr, rr)
            del c_h, r_h, c_d, r_d
        finally:
            ph.phprng_destroy(a)
            ph.phprng_destroy(b)


@pytest.mark.parametrize("width,count,per,want_c", [(32, 1500, 4096, True), (32, 37, 1001, True),
                                                    (32, 64, 777, False), (64, 20, 513, True)],
                         ids=["whole_vec", "ragged", "r_only_ragged", "wide64"])
def test_pinned_host_outputs(ph, torch, width, count, per, want_c):
    """Pinned host outputs only: same bytes as device outputs, ragged lengths
    included, and the streams continue from there."""
    inst = workloads.draw_instances(count, width=width, seed=77 + count)
    a = ph.phprng_create(width, inst, 0)
    b = ph.phprng_create(width, inst, 0)
    try:
        cdt = torch.int32 if width == 32 else torch.int64
        for _ in range(2):
            c_h = torch.zeros(count * per, dtype=cdt, pin_memory=True) if want_c else None
            r_h = torch.zeros(count * per, dtype=torch.float64, pin_memory=True)
            ph.phprng_generate(a, 0, count, per, c_h, r_h, None)
            c_d, r_d = generate(ph, torch, b, width, 0, count, per)
            if want_c:
                got = c_h.numpy().view(np.uint32 if width == 32 else np.uint64)
                assert np.array_equal(got.reshape(count, per).astype(np.uint64), c_d)
            assert np.array_equal(r_h.numpy().reshape(count, per).view(np.uint64),
                                  r_d.view(np.uint64))
        orc = OracleStreams(inst)
        k = min(count, 3)
        cr, rr = orc.next(0, k, 2 * per)
        assert_same(c_d[:k], r_d[:k], cr[:, per:], rr[:, per:])
    finally:
        ph.phprng_destroy(a)
        ph.phprng_destroy(b)


def test_launch_order_over_ranges(ph, torch):
    """Launches of 1,024 instances or more run them heaviest program first
    (32-bit before 64-bit): outputs stay instance-major and states right over
    whole-table, sub-range, repeated and short ranges of a shuffled mixed
    table."""
    i32 = workloads.draw_instances(2600, seed=91)
    i64 = workloads.draw_instances(500, width=64, seed=92)
    cat = workloads.concat_instances(i32, i64)
    perm = np.random.default_rng(93).permutation(3100)
    mixed = {k: v[perm] for k, v in cat.items()}
    ctx = ph.phprng_create(0, mixed, 0)
    try:
        orc = OracleStreams(mixed)
        pos = np.zeros(3100, dtype=np.int64)
        for first, num, per in [(0, 3100, 40), (300, 2600, 33), (300, 2600, 5), (0, 1024, 8),
                                (0, 3100, 17), (5, 100, 9), (2000, 1100, 12)]:
            c, r = generate(ph, torch, ctx, 0, first, num, per)
            assert_same(c, r, *orc.next(first, num, per))
            pos[first:first + num] += per
        check_state(ph, ctx, orc, 0, 3100, pos)
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("n32,n64,calls", [(3, 0, [100003, 5000, 2048, 2047]),
                                            (2, 2, [50001, 4096, 1]),
                                            (1, 0, [1 << 22])],
                         ids=["32bit_ragged", "mixed", "one_instance_4M"])
def test_split_launches(ph, torch, n32, n64, calls):
    """Calls with few instances cut every instance into chunks whose start
    message comes from a pre-pass of skip sums: outputs, continuation and
    states equal the oracle's stream, for ragged and chunk-sized lengths."""
    tables = [workloads.draw_instances(n32, seed=501 + n32)]
    if n64:
        tables.append(workloads.draw_instances(n64, width=64, seed=601 + n64))
    inst = workloads.concat_instances(*tables)
    count = n32 + n64
    width = 32 if n64 == 0 else 0
    ctx = ph.phprng_create(width, inst, 0)
    try:
        orc = OracleStreams(inst)
        for per in calls:
            c, r = generate(ph, torch, ctx, width, 0, count, per)
            assert_same(c, r, *orc.next(0, count, per))
        check_state(ph, ctx, orc, 0, count, [sum(calls)] * count)
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("exps,calls", [((3, 5, 9, 17), (4096, 1001, 3, 100003)),
                                        ((3, 5, 9, 17, 65537, None), (4096, 1001, 3))],
                         ids=["light_programs", "mixed_with_random"])
def test_small_exponents(ph, torch, exps, calls):
    """The paper's small exponents (e = 3, 5, 9, 17), alone (the launches take
    the light-program instantiation, the long call a split launch) and mixed
    with 65537 and random exponents: ragged calls and continuation against
    the oracle."""
    tables = [workloads.draw_instances(6, seed=700 + (e or 99), exponent=e) for e in exps]
    inst = workloads.concat_instances(*tables)
    count = len(inst["n"])
    ctx = ph.phprng_create(32, inst, 0)
    try:
        orc = OracleStreams(inst)
        for per in calls:
            c, r = generate(ph, torch, ctx, 32, 0, count, per)
            assert_same(c, r, *orc.next(0, count, per))
        check_state(ph, ctx, orc, 0, count, [sum(calls)] * count)
    finally:
        ph.phprng_destroy(ctx)
    if exps[-1] is not None:
        return
    tables = [workloads.draw_instances(3, width=64, seed=720 + e, exponent=e) for e in (3, 17, 65537)]
    tables.append(workloads.draw_instances(3, width=64, seed=799))
    inst = workloads.concat_instances(*tables)
    ctx = ph.phprng_create(64, inst, 0)
    try:
        orc = OracleStreams(inst)
        for per in (1000, 129):
            c, r = generate(ph, torch, ctx, 64, 0, 12, per)
            assert_same(c, r, *orc.next(0, 12, per))
    finally:
        ph.phprng_destroy(ctx)


def test_small_exponent_full_size_sampled(ph, torch):
    """65,536 instances with e = 9 x 4,096 numbers (the small-exponent bench
    launch): sampled instances against the oracle, R on every number."""
    inst = workloads.workload_instances("plain32_e9_65536x4096")
    N, per = 65536, 4096
    assert np.all(inst["e"] == 9)
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        c, r = generate(ph, torch, ctx, 32, 0, N, per)
        sample = np.unique(np.concatenate([[0, 1, N - 1], np.random.default_rng(9).choice(N, 61)]))
        rows = workloads.instance_rows(inst)[sample]
        cr, rr, _, _ = oracle.generate_many(rows, per, threads=THREADS)
        assert_same(c[sample], r[sample], cr, rr)
        n1 = (inst["n"] + np.uint64(1)).astype(np.float64)[:, None]
        ref = (c + np.uint64(1)).astype(np.float64) / n1     # both exact in double: RN quotient
        assert np.array_equal(ref.view(np.uint64), r.view(np.uint64))
    finally:
        ph.phprng_destroy(ctx)


def test_plain32_full_size_first_call_and_64_calls(ph, torch):
    """65,536 instances x 4,096 numbers per call, the benchmark's launch:
    the whole first call against the oracle, then 63 more R-only calls and
    the states plus the last call's outputs of sampled instances."""
    name = "plain32_65536x4096x64"
    w = workloads.WORKLOADS[name]
    inst = workloads.workload_instances(name)
    N, per = w["instances"], w["per_inst"]
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        orc = OracleStreams(inst)
        c, r = generate(ph, torch, ctx, 32, 0, N, per)
        assert_same(c, r, *orc.next(0, N, per))
        del c, r
        rbuf = torch.empty(N * per, dtype=torch.float64, device="cuda")
        for call in range(62):
            ph.phprng_generate(ctx, 0, N, per, None, rbuf, None)
        c, r = generate(ph, torch, ctx, 32, 0, N, per)
        rng = np.random.default_rng(64)
        sample = np.unique(np.concatenate([[0, N - 1], rng.choice(N, 254, replace=False)]))
        rows = orc.rows[sample].copy()
        _, _, st, _ = oracle.generate_many(rows, 62 * per, threads=THREADS, want_c=False,
                                           want_r=False)
        rows[:, 4:6] = st
        cr, rr, st2, _ = oracle.generate_many(rows, per, threads=THREADS)
        assert_same(c[sample], r[sample], cr, rr)
        for j, i in enumerate(sample):
            s = ph.phprng_get_state(ctx, int(i))
            assert (s["m"], s["s"], s["pos"]) == (int(st2[j, 0]), int(st2[j, 1]), 64 * per)
        # property on every number of the last call: R is the rounded (c+1)/(n+1)
        n = inst["n"].astype(np.float64)[:, None]
        ref = (c + np.uint64(1)).astype(np.float64) / (n + 1.0)
        assert np.array_equal(ref.view(np.uint64), r.view(np.uint64))
        assert np.all(c < inst["n"][:, None])
    finally:
        ph.phprng_destroy(ctx)


def test_wide64_chunk_sampled(ph, torch):
    """4,096 64-bit safe primes x 2^16 numbers (one chunk of the 2^20-number
    workload): sampled instances against the oracle, properties on all."""
    name = "wide64_4096x2^20"
    inst = workloads.workload_instances(name)
    N, per = 4096, 1 << 16
    ctx = ph.phprng_create(64, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        orc = OracleStreams(inst)
        c, r = generate(ph, torch, ctx, 64, 0, N, per)
        sample = np.unique(np.concatenate([[0, N - 1], np.random.default_rng(7).choice(N, 30)]))
        rows = orc.rows[sample].copy()
        cr, rr, st, _ = oracle.generate_many(rows, per, threads=THREADS)
        assert_same(c[sample], r[sample], cr, rr)
        n = inst["n"][:, None]
        assert np.all(c < n)
        ref = (c + np.uint64(1)).astype(np.float64) / (n + np.uint64(1)).astype(np.float64)
        assert np.array_equal(ref.view(np.uint64), r.view(np.uint64))
        for j, i in enumerate(sample[:5]):
            s = ph.phprng_get_state(ctx, int(i))
            assert (s["m"], s["s"]) == (int(st[j, 0]), int(st[j, 1]))
    finally:
        ph.phprng_destroy(ctx)


def test_repeatable(ph, torch):
    inst = workloads.draw_instances(33, seed=9)
    outs = []
    for _ in range(2):
        ctx = ph.phprng_create(32, inst, 0)
        outs.append(generate(ph, torch, ctx, 32, 0, 33, 777))
        ph.phprng_destroy(ctx)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1].view(np.uint64), outs[1][1].view(np.uint64))


def test_argument_errors_on_device(ph, torch):
    inst = workloads.draw_instances(4, seed=3)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        r = torch.empty(16, dtype=torch.float64, device="cuda")
        with pytest.raises(ph.PhprngError) as ei:
            ph.phprng_generate(ctx, 3, 2, 4, None, r)            # range past the table
        assert ei.value.status == ph.PHPRNG_EINVAL
        with pytest.raises(ph.PhprngError):
            ph.phprng_generate(ctx, 0, 1, 4, None, r.data_ptr() + 4)   # misaligned
        with pytest.raises(ph.PhprngError):
            ph.phprng_generate(ctx, 0, 1, 4, None, None)          # no output
        ph.phprng_generate(ctx, 0, 4, 0, None, r)                 # per_inst = 0: no-op
        ph.phprng_generate(ctx, 2, 0, 4, None, r)                 # num_inst = 0: no-op
        ph.phprng_generate(ctx, 4, 0, 4, None, r)                 # empty range at the table's end
        assert all(ph.phprng_get_state(ctx, i)["pos"] == 0 for i in range(4))
        with pytest.raises(ph.PhprngError):
            ph.phprng_get_state(ctx, 4)
    finally:
        ph.phprng_destroy(ctx)


def test_maximum_length_single_call(ph, torch):
    """One stream of 2^32 + 777 numbers in one call (c only, 17 GB): indices
    past 2^31 and 2^32 inside one launch (split into chunks).  Sampled runs of
    8 numbers at positions across the call equal the oracle's, each started
    from the state its own prefix table gives by Eq. 7, and the final state
    is the oracle's state after 2^32 + 777 steps."""
    inst = workloads.draw_instances(1, seed=77)
    n, e, m0, s0 = (int(inst[k][0]) for k in ("n", "e", "m0", "s0"))
    per = (1 << 32) + 777
    table = oracle.PrefixTable(P31, A31, 1 << 16)
    L0 = int(oracle.dlog(P31, A31, [s0])[0])
    ctx = ph.phprng_create(32, inst, 0)
    try:
        c = torch.empty(per, dtype=torch.int32, device="cuda")
        ph.phprng_generate(ctx, 0, 1, per, c, None)
        torch.cuda.synchronize()
        for t in (0, 1, 4095, (1 << 31) - 3, (1 << 31) + 5, (1 << 32) - 5, 1 << 32, per - 8):
            m_t, s_t = table.state_at(n, m0, L0, t)
            want, _, _ = oracle.generate(n, e, P31, A31, m_t, s_t, 8)
            got = c[t:t + 8].cpu().numpy().view(np.uint32).astype(np.uint64)
            assert np.array_equal(got, want), t
        st = ph.phprng_get_state(ctx, 0)
        assert (st["m"], st["s"], st["pos"]) == (*table.state_at(n, m0, L0, per), per)
        del c
    finally:
        ph.phprng_destroy(ctx)
