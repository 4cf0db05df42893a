"""GPU tests of the serving loop through the C ABI: every served request
against the oracle at the position the server gave it (so each result is the
same as alone), FIFO positions per stream, admission bounded by the output
budget, streams' states after shutdown, and refusal of oversize requests."""
import os
import time

import numpy as np
import pytest

import oracle
from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu
P31, A31 = 2147483647, 784588716


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def table31():
    return oracle.PrefixTable(P31, A31, 1 << 16)


def drain(ph, srv, total, copy=True, release=True, timeout=60.0):
    got = []
    t0 = time.time()
    while len(got) < total:
        assert time.time() - t0 < timeout, "server did not finish in time"
        comp = ph.phprng_server_poll(srv, 4096, 20_000_000)
        for c in comp:
            rec = dict(id=int(c["id"]), tag=int(c["tag"]), inst=int(c["inst"]),
                       start=int(c["start"]), len=int(c["len"]),
                       arrival=int(c["arrival_ns"]), done=int(c["done_ns"]))
            if copy:
                r = np.empty(rec["len"], dtype=np.float64)
                cc = np.empty(rec["len"], dtype=np.uint32)
                ph.phprng_server_copy(srv, rec["id"], r, cc)
                rec["r"], rec["c"] = r, cc
            got.append(rec)
        if release and len(comp):
            ph.phprng_server_release(srv, comp["id"])
    return got


@pytest.mark.parametrize("tile", [1024, 0], ids=["tile1024", "auto_tile"])
def test_served_requests_match_oracle_and_fifo(ph, torch, table31, tile):
    inst = workloads.draw_instances(40, seed=601)
    L0 = oracle.dlog(P31, A31, inst["s0"])
    ctx = ph.phprng_create(32, inst, 0)
    srv = ph.phprng_server_create(ctx, 64 << 20, inflight=3, tile=tile, want_c=1)
    try:
        rng = np.random.default_rng(3)
        n = 400
        streams = rng.integers(0, 40, n)
        lens = np.minimum(np.round(np.exp(rng.normal(np.log(300), 1.5, n))).astype(np.int64) + 1,
                          20000)
        t0 = ph.phprng_clock_ns() + 5_000_000
        arrivals = t0 + np.sort(rng.integers(0, 80_000_000, n))        # 80 ms of arrivals
        first = ph.phprng_server_submit(srv, streams, lens, np.arange(n), arrivals)
        got = drain(ph, srv, n)
        st = ph.phprng_server_stats_get(srv)
        assert st["completed"] == n and st["batches"] >= 2
    finally:
        ph.phprng_server_destroy(srv)
    try:
        by_tag = {g["tag"]: g for g in got}
        cursor = {}
        for k in range(n):                               # FIFO positions per stream
            g = by_tag[k]
            i = int(streams[k])
            assert g["inst"] == i and g["len"] == int(lens[k]) and g["id"] == first + k
            assert g["start"] == cursor.get(i, 0)
            cursor[i] = g["start"] + g["len"]
            assert g["done"] >= g["arrival"] >= int(arrivals[k])
        for g in got:                                    # each result is the stream's own numbers
            m, s = table31.state_at(int(inst["n"][g["inst"]]), int(inst["m0"][g["inst"]]),
                                    int(L0[g["inst"]]), g["start"])
            c, r, _ = oracle.generate(int(inst["n"][g["inst"]]), int(inst["e"][g["inst"]]),
                                      P31, A31, m, s, g["len"])
            assert np.array_equal(g["c"].astype(np.uint64), c), g["tag"]
            assert np.array_equal(g["r"].view(np.uint64), r.view(np.uint64)), g["tag"]
        for i, pos in cursor.items():                    # stored state after shutdown
            s = ph.phprng_get_state(ctx, i)
            m, sk = table31.state_at(int(inst["n"][i]), int(inst["m0"][i]), int(L0[i]), pos)
            assert (s["m"], s["s"], s["pos"]) == (m, sk, pos)
    finally:
        ph.phprng_destroy(ctx)


def test_admission_is_bounded_by_the_budget(ph, torch):
    inst = workloads.draw_instances(8, seed=602)
    ctx = ph.phprng_create(32, inst, 0)
    budget = 64 * 1024                                   # 8,192 doubles
    srv = ph.phprng_server_create(ctx, budget, inflight=2, tile=512)
    try:
        n = 200
        lens = np.full(n, 3000)                          # 24 KB each: two fit at a time
        ph.phprng_server_submit(srv, np.arange(n) % 8, lens)
        seen_max = 0
        got = []
        t0 = time.time()
        while len(got) < n:
            assert time.time() - t0 < 60
            st = ph.phprng_server_stats_get(srv)
            seen_max = max(seen_max, st["outstanding_bytes"])
            comp = ph.phprng_server_poll(srv, 16, 10_000_000)
            got.extend(int(x) for x in comp["id"])
            if len(comp):
                ph.phprng_server_release(srv, comp["id"])
        st = ph.phprng_server_stats_get(srv)
        assert seen_max <= budget and st["max_waiting"] > 0 and st["completed"] == n
        with pytest.raises(ph.PhprngError) as ei:
            ph.phprng_server_submit(srv, [0], [budget])   # more than the whole arena
        assert ei.value.status == ph.PHPRNG_EBUDGET
        with pytest.raises(ph.PhprngError):
            ph.phprng_generate(ctx, 0, 1, 4, None, torch.empty(4, dtype=torch.float64,
                                                               device="cuda"))
    finally:
        ph.phprng_server_destroy(srv)
        ph.phprng_destroy(ctx)


def test_mixed_width_serving(ph, torch, table31):
    i32 = workloads.draw_instances(6, seed=603)
    i64 = workloads.draw_instances(3, width=64, seed=604)
    inst = workloads.concat_instances(i32, i64)
    L0 = oracle.dlog(P31, A31, inst["s0"])
    ctx = ph.phprng_create(0, inst, 0)
    srv = ph.phprng_server_create(ctx, 8 << 20, tile=256)
    try:
        streams = np.array([0, 8, 3, 7, 8, 0, 6, 2])
        lens = np.array([100, 333, 1, 4096, 10, 77, 5000, 640])
        ph.phprng_server_submit(srv, streams, lens, np.arange(8))
        got = drain(ph, srv, 8, copy=False, release=False)
        for g in got:
            r = np.empty(g["len"], dtype=np.float64)
            ph.phprng_server_copy(srv, g["id"], r)
            i = g["inst"]
            m, s = table31.state_at(int(inst["n"][i]), int(inst["m0"][i]), int(L0[i]), g["start"])
            _, rr, _ = oracle.generate(int(inst["n"][i]), int(inst["e"][i]), P31, A31, m, s,
                                       g["len"])
            assert np.array_equal(r.view(np.uint64), rr.view(np.uint64))
    finally:
        ph.phprng_server_destroy(srv)
        ph.phprng_destroy(ctx)


def test_served_unit_and_constant_skip_streams_match_oracle(ph, torch):
    """A server over constant-skip streams (a = 1: s_k = s0 = b for every k;
    b = 1 is the unit skip): each served request starts at m0 + start b
    (Eq. 3 summed) and equals the oracle's Eq. 9 from there, and the streams'
    states after shutdown follow."""
    inst = workloads.draw_instances(12, seed=611)
    rows = workloads.instance_rows(inst).copy()
    rows[:, 2], rows[:, 3] = 65537, 1                  # one skip generator per context
    rows[:, 5] = np.arange(1, 13) * 5000
    rows[:6, 5] = 1                                    # unit skip (b = 1) for the first six
    ctx = ph.phprng_create(32, rows, ph.PHPRNG_ALLOW_SHARED_N)
    srv = ph.phprng_server_create(ctx, 16 << 20, inflight=2, tile=0, want_c=1)
    try:
        rng = np.random.default_rng(9)
        n = 60
        streams = rng.integers(0, 12, n)
        lens = rng.integers(1, 3000, n)
        t0 = ph.phprng_clock_ns() + 2_000_000
        arrivals = t0 + np.sort(rng.integers(0, 20_000_000, n))
        ph.phprng_server_submit(srv, streams, lens, np.arange(n), arrivals)
        got = drain(ph, srv, n)
    finally:
        ph.phprng_server_destroy(srv)
    try:
        for g in got:
            n_, e, p, a, m0, b = (int(x) for x in rows[g["inst"]])
            oc, orr, _ = oracle.generate(n_, e, p, a, (m0 + g["start"] * b) % n_, b, g["len"])
            assert np.array_equal(g["c"].astype(np.uint64), oc)
            assert np.array_equal(g["r"].view(np.uint64), orr.view(np.uint64))
        total = {}
        for k in range(n):
            total[int(streams[k])] = total.get(int(streams[k]), 0) + int(lens[k])
        for i, t in total.items():
            s = ph.phprng_get_state(ctx, i)
            n_, b, m0 = int(rows[i, 0]), int(rows[i, 5]), int(rows[i, 4])
            assert s["pos"] == t and s["m"] == (m0 + t * b) % n_ and s["s"] == b
    finally:
        ph.phprng_destroy(ctx)
