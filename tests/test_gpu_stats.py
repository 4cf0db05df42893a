"""GPU tests of the fused consumer mode: per-stream exact sums, histogram and
adjacent-stream product sums reduced on chip, against the oracle's
definitions on the oracle's own ciphertexts (integers exact, doubles 0 ULP)."""
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


def run_stats(ph, torch, ctx, first, num, per, want_c=False, want_r=False):
    sb = torch.empty(num * ph.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    c = torch.empty(num * per, dtype=torch.int32, device="cuda") if want_c else None
    r = torch.empty(num * per, dtype=torch.float64, device="cuda") if want_r else None
    ph.phprng_generate(ctx, first, num, per, c, r, sb)
    torch.cuda.synchronize()
    st = sb.cpu().numpy().view(ph.STATS_DTYPE)
    cn = c.cpu().numpy().view(np.uint32).astype(np.uint64).reshape(num, per) if want_c else None
    rn = r.cpu().numpy().reshape(num, per) if want_r else None
    return st, cn, rn


def u128(lo, hi):
    return int(lo) | (int(hi) << 64)


def check_stats(st, c_ref, ns, idx=None):
    """st: device stats rows for instances idx (all when None); c_ref: oracle c
    for every instance of the call (num, per); ns: moduli of the call."""
    num = c_ref.shape[0]
    for j in (range(num) if idx is None else idx):
        X, Y, hist, mean, var = oracle.stats(c_ref[j], int(ns[j]))
        row = st[j]
        assert u128(row["x_lo"], row["x_hi"]) == X, j
        assert u128(row["y_lo"], row["y_hi"]) == Y, j
        assert np.array_equal(row["hist"], hist), j
        assert row["count"] == c_ref.shape[1]
        assert row["mean"].view(np.uint64) == np.float64(mean).view(np.uint64), j
        assert row["var"].view(np.uint64) == np.float64(var).view(np.uint64), j
        if j + 1 < num:
            Z, corr = oracle.corr(c_ref[j], c_ref[j + 1], int(ns[j]), int(ns[j + 1]))
        else:
            Z, corr = 0, 0.0
        assert u128(row["z_lo"], row["z_hi"]) == Z, j
        assert row["corr"].view(np.uint64) == np.float64(corr).view(np.uint64), j


@pytest.mark.parametrize("num,per", [(1, 1), (3, 2), (20, 100), (17, 4097), (9, 128), (33, 1000)])
def test_stats_match_oracle(ph, torch, num, per):
    inst = workloads.draw_instances(num + 3, seed=300 + num + per)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        rows = workloads.instance_rows(inst)
        first = 2 if num + 2 <= len(rows) else 0
        c_ref, _, _, _ = oracle.generate_many(rows[first:first + num], per, threads=THREADS)
        st, _, _ = run_stats(ph, torch, ctx, first, num, per)
        check_stats(st, c_ref, inst["n"][first:first + num])
        # the streams advanced exactly as a plain call would
        _, _, srow, _ = oracle.generate_many(rows[first:first + num], per, threads=THREADS)
        for j in range(num):
            s = ph.phprng_get_state(ctx, first + j)
            assert (s["m"], s["s"], s["pos"]) == (int(srow[j, 0]), int(srow[j, 1]), per)
    finally:
        ph.phprng_destroy(ctx)


def test_stats_with_outputs_and_host_stats(ph, torch):
    inst = workloads.draw_instances(12, seed=311)
    a = ph.phprng_create(32, inst, 0)
    b = ph.phprng_create(32, inst, 0)
    try:
        per = 777
        rows = workloads.instance_rows(inst)
        c_ref, r_ref, _, _ = oracle.generate_many(rows, per, threads=THREADS)
        st, c, r = run_stats(ph, torch, a, 0, 12, per, want_c=True, want_r=True)
        assert np.array_equal(c, c_ref)
        assert np.array_equal(r.view(np.uint64), r_ref.view(np.uint64))
        check_stats(st, c_ref, inst["n"])
        host = np.zeros(12, dtype=ph.STATS_DTYPE)                  # host statistics buffer
        ph.phprng_generate(b, 0, 12, per, None, None, host)
        assert host.tobytes() == st.tobytes()
    finally:
        ph.phprng_destroy(a)
        ph.phprng_destroy(b)


def test_stats_full_period_closed_forms(ph, torch):
    """Whole period of a tiny instance: X, Y and the histogram are fixed by
    the uniformity of the period (every c exactly p-1 times)."""
    from test_gpu_parity import primitive_root
    n, p, e = 1019, 509, 7
    a = primitive_root(p)
    inst = {"n": [n], "e": [e], "p": [p], "a": [a], "m0": [3], "s0": [1]}
    ctx = ph.phprng_create(32, inst, 0)
    try:
        P = n * (p - 1)
        st, _, _ = run_stats(ph, torch, ctx, 0, 1, P)
        row = st[0]
        assert u128(row["x_lo"], row["x_hi"]) == (p - 1) * n * (n + 1) // 2
        assert u128(row["y_lo"], row["y_hi"]) == (p - 1) * n * (n + 1) * (2 * n + 1) // 6
        expect = np.zeros(256, dtype=np.int64)
        for cc in range(n):
            expect[(256 * (cc + 1)) // (n + 1)] += p - 1
        assert np.array_equal(row["hist"].astype(np.int64), expect)
        assert row["mean"] == 0.5
    finally:
        ph.phprng_destroy(ctx)


def test_stats_full_size_sampled(ph, torch):
    """The 65,536 x 4,096 workload in fused mode: sampled streams (block edges
    included) against the oracle, histogram totals on all streams."""
    name = "plain32_65536x4096x64"
    inst = workloads.workload_instances(name)
    N, per = 65536, 4096
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        st, _, _ = run_stats(ph, torch, ctx, 0, N, per)
        assert np.all(st["hist"].sum(axis=1) == per)
        assert np.all(st["count"] == per)
        rng = np.random.default_rng(3)
        pick = sorted(set([0, 6, 7, 8, 15, 16, N - 9, N - 8, N - 2, N - 1] +
                          [int(x) for x in rng.choice(N - 1, 40, replace=False)]))
        rows = workloads.instance_rows(inst)
        need = sorted(set(pick + [j + 1 for j in pick if j + 1 < N]))
        c_need, _, _, _ = oracle.generate_many(rows[need], per, threads=THREADS)
        cmap = {j: c_need[k] for k, j in enumerate(need)}
        for j in pick:
            X, Y, hist, mean, var = oracle.stats(cmap[j], int(inst["n"][j]))
            row = st[j]
            assert (u128(row["x_lo"], row["x_hi"]), u128(row["y_lo"], row["y_hi"])) == (X, Y)
            assert np.array_equal(row["hist"], hist)
            assert row["var"].view(np.uint64) == np.float64(var).view(np.uint64)
            if j + 1 < N:
                Z, corr = oracle.corr(cmap[j], cmap[j + 1], int(inst["n"][j]),
                                      int(inst["n"][j + 1]))
                assert u128(row["z_lo"], row["z_hi"]) == Z, j
                assert row["corr"].view(np.uint64) == np.float64(corr).view(np.uint64), j
    finally:
        ph.phprng_destroy(ctx)


def test_stats_rejects_64bit(ph, torch):
    inst = workloads.draw_instances(2, width=64, seed=5)
    ctx = ph.phprng_create(64, inst, 0)
    try:
        sb = torch.empty(2 * ph.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        with pytest.raises(ph.PhprngError):
            ph.phprng_generate(ctx, 0, 2, 10, None, None, sb)
    finally:
        ph.phprng_destroy(ctx)
