"""GPU tests of the batched persistent launch (plans) through the C ABI:
mixed 32/64-bit instances, uneven lengths, start offsets reached by Eq. 7,
CONTINUE chains; each request against the oracle, the same alone and in the
mix, the same for plain, graph and every autotuned configuration."""
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


def oracle_request(table31, inst, L0, i, start, length):
    n, e = int(inst["n"][i]), int(inst["e"][i])
    m, s = table31.state_at(n, int(inst["m0"][i]), int(L0[i]), start)
    c, r, st = oracle.generate(n, e, P31, A31, m, s, length)
    return c, r, st


def run_plan(ph, torch, ctx, reqs, total, mode="plain", tile=0):
    c = torch.zeros(max(total, 1), dtype=torch.int64, device="cuda")
    r = torch.zeros(max(total, 1), dtype=torch.float64, device="cuda")
    plan = ph.phprng_plan_create(ctx, reqs, tile)
    try:
        if mode == "plain":
            ph.phprng_plan_launch(plan, c, r, ctx=ctx)
        elif mode == "graph":
            ph.phprng_plan_launch_graph(plan, c, r, ctx=ctx)
            ph.phprng_plan_launch_graph(plan, c, r, ctx=ctx)
        else:
            ph.phprng_plan_autotune(plan, c, r, ctx=ctx)
            ph.phprng_plan_launch(plan, c, r, ctx=ctx)
        torch.cuda.synchronize()
    finally:
        ph.phprng_plan_destroy(plan)
    return c.cpu().numpy().view(np.uint64), r.cpu().numpy()


@pytest.fixture(scope="module")
def mixed(ph):
    i32 = workloads.draw_instances(12, seed=501)
    i64 = workloads.draw_instances(5, width=64, seed=502)
    inst = workloads.concat_instances(i32, i64)
    L0 = oracle.dlog(P31, A31, inst["s0"])
    rng = np.random.default_rng(5)
    reqs, off = [], 0
    lens = [1, 2, 31, 128, 129, 1000, 4097, 20000, 70000, 0, 3, 17, 5000, 64, 77, 100000, 9]
    for i in range(17):
        ln = lens[i]
        reqs.append((i, int(rng.integers(0, 1 << 40)), ln, off, off))
        off += ln
    # CONTINUE chains: instance 3 (32-bit) and 14 (64-bit) get two more requests each
    C = ph.PHPRNG_CONTINUE
    for i, ln in ((3, 500), (14, 700), (3, 33), (14, 1)):
        reqs.append((i, C, ln, off, off))
        off += ln
    return inst, L0, reqs, off


def expected(table31, inst, L0, reqs):
    cursor = {}
    out = []
    for (i, offset, ln, co, ro) in reqs:
        if ln == 0:                                   # ignored by the library
            continue
        start = cursor.get(i, 0) if offset == 2 ** 64 - 1 else offset
        cursor[i] = start + ln
        c, r, st = oracle_request(table31, inst, L0, i, start, ln)
        out.append((co, ro, ln, c, r))
    return out, cursor


@pytest.mark.parametrize("mode,tile", [("plain", 0), ("plain", 96), ("graph", 0), ("tuned", 0)])
def test_mixed_batch_matches_oracle(ph, torch, table31, mixed, mode, tile):
    inst, L0, reqs, total = mixed
    ctx = ph.phprng_create(0, inst, 0)
    try:
        c, r = run_plan(ph, torch, ctx, reqs, total, mode, tile)
        exp, cursor = expected(table31, inst, L0, reqs)
        for k, (co, ro, ln, ce, re) in enumerate(exp):
            assert np.array_equal(c[co:co + ln], ce), k
            assert np.array_equal(r[ro:ro + ln].view(np.uint64), re.view(np.uint64)), k
        # every touched instance now sits at the end of its last request
        for i, pos in cursor.items():
            s = ph.phprng_get_state(ctx, i)
            assert s["pos"] == pos
            m, sk = table31.state_at(int(inst["n"][i]), int(inst["m0"][i]), int(L0[i]), pos)
            assert (s["m"], s["s"]) == (m, sk)
    finally:
        ph.phprng_destroy(ctx)


def test_alone_equals_in_the_mix(ph, torch, table31, mixed):
    inst, L0, reqs, total = mixed
    ctx = ph.phprng_create(0, inst, 0)
    try:
        c_mix, r_mix = run_plan(ph, torch, ctx, reqs, total)
        for k, (i, offset, ln, co, ro) in enumerate(reqs):
            if offset == ph.PHPRNG_CONTINUE or ln == 0:
                continue
            c1, r1 = run_plan(ph, torch, ctx, [(i, offset, ln, 0, 0)], ln)
            assert np.array_equal(c1[:ln], c_mix[co:co + ln]), k
            assert np.array_equal(r1[:ln].view(np.uint64), r_mix[ro:ro + ln].view(np.uint64)), k
    finally:
        ph.phprng_destroy(ctx)


def test_batch_then_generate_continues(ph, torch, table31):
    inst = workloads.draw_instances(6, seed=503)
    L0 = oracle.dlog(P31, A31, inst["s0"])
    ctx = ph.phprng_create(32, inst, 0)
    try:
        reqs = [(i, 1000 * i + 7, 300 + i, 400 * i, 400 * i) for i in range(6)]
        run_plan(ph, torch, ctx, reqs, 2400)
        c = torch.empty(6 * 50, dtype=torch.int32, device="cuda")
        ph.phprng_generate(ctx, 0, 6, 50, c, None)
        c = c.cpu().numpy().view(np.uint32).reshape(6, 50)
        for i in range(6):
            ce, _, _ = oracle_request(table31, inst, L0, i, 1000 * i + 7 + 300 + i, 50)
            assert np.array_equal(c[i].astype(np.uint64), ce)
    finally:
        ph.phprng_destroy(ctx)


def test_generate_batch_one_shot_and_errors(ph, torch, table31):
    inst = workloads.draw_instances(4, seed=504)
    L0 = oracle.dlog(P31, A31, inst["s0"])
    ctx = ph.phprng_create(32, inst, 0)
    try:
        r = torch.zeros(1000, dtype=torch.float64, device="cuda")
        ph.phprng_generate_batch(ctx, [(2, 12345, 1000, 0, 0)], None, r)
        _, re, _ = oracle_request(table31, inst, L0, 2, 12345, 1000)
        assert np.array_equal(r.cpu().numpy().view(np.uint64), re.view(np.uint64))
        with pytest.raises(ph.PhprngError):
            ph.phprng_plan_create(ctx, [(4, 0, 1, 0, 0)])          # instance out of range
        with pytest.raises(ph.PhprngError):
            ph.phprng_plan_create(ctx, [(0, 2 ** 64 - 2, 5, 0, 0)])  # position overflow
    finally:
        ph.phprng_destroy(ctx)


def test_batched_workload_sampled(ph, torch, table31):
    """A reduced batched workload (1,000 instances, 80 % 32-bit, lengths
    log-uniform up to 2^16, offsets up to 2^40): sampled requests vs oracle."""
    i32 = workloads.draw_instances(800, seed=505)
    i64 = workloads.draw_instances(200, width=64, seed=506)
    inst = workloads.concat_instances(i32, i64)
    reqs = workloads.batched_requests(800, 200, max_len=1 << 16, seed=507)
    total = int(reqs["len"].sum())
    L0 = oracle.dlog(P31, A31, inst["s0"])
    ctx = ph.phprng_create(0, inst, 0)
    try:
        c, r = run_plan(ph, torch, ctx, reqs, total, "tuned")
        rng = np.random.default_rng(9)
        for k in sorted(set([0, 799, 800, 999] + [int(x) for x in rng.choice(1000, 24)])):
            i, offset, ln, co, ro = (int(x) for x in reqs[k])
            ce, re, _ = oracle_request(table31, inst, L0, i, offset, ln)
            assert np.array_equal(c[co:co + ln], ce), k
            assert np.array_equal(r[ro:ro + ln].view(np.uint64), re.view(np.uint64)), k
    finally:
        ph.phprng_destroy(ctx)
