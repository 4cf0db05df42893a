"""GPU tests of the serial-test consumer (Tests section, items 1-5) through the
C ABI: the pooled D-tuple histograms must equal the oracle's exactly, and the
streams must continue as after phprng_generate."""
import os

import numpy as np
import pytest

import oracle
from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
PAPER_SIZES = [(1, 1 << 20), (2, 1 << 10), (3, 100), (4, 32), (5, 16)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def oracle_hist(_unused, start_rows, per, D, B):
    """Histogram of per numbers of every stream from its current state."""
    c, _, st, _ = oracle.generate_many(start_rows, per, threads=THREADS, want_r=False)
    h = np.zeros(B ** D, dtype=np.uint64)
    for k in range(len(start_rows)):
        oracle.serial_hist(c[k], int(start_rows[k, 0]), D, B, h)
    return h, st


@pytest.mark.parametrize("D,B", PAPER_SIZES + [(7, 8), (3, 2), (1, 10), (2, 14), (1, 224), (1, 225)])
def test_serial_histograms_match_oracle(ph, torch, D, B):
    """Two consecutive calls (ragged lengths, tuples spanning lanes and warp
    groups), histograms accumulated on the device, states continued.  Up to
    224 bins the kernel counts in shared memory (225: the device histogram)."""
    inst = workloads.draw_instances(37, seed=90 + D)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        rows = workloads.instance_rows(inst).copy()
        hist = torch.zeros(B ** D, dtype=torch.int64, device="cuda")
        want = np.zeros(B ** D, dtype=np.uint64)
        for per in (1001, 4099):
            ph.phprng_serial_test(ctx, 0, 37, per, D, B, hist)
            h, st = oracle_hist(None, rows, per, D, B)
            want += h
            rows[:, 4:6] = st
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
        for i in (0, 17, 36):
            s = ph.phprng_get_state(ctx, i)
            assert (s["m"], s["s"], s["pos"]) == (int(rows[i, 4]), int(rows[i, 5]), 5100)
    finally:
        ph.phprng_destroy(ctx)


def test_serial_at_scale_and_chi_square(ph, torch):
    """4,096 streams x 65,536 numbers, D = 2 and the paper's 2^20 bins: equal
    to the oracle, and the chi-square of the pooled histogram is unremarkable
    (|z| < 6 against the uniform expectation)."""
    inst = workloads.draw_instances(4096, seed=93)
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        D, B, per = 2, 1 << 10, 1 << 16
        hist = torch.zeros(B ** D, dtype=torch.int64, device="cuda")
        ph.phprng_serial_test(ctx, 0, 4096, per, D, B, hist)
        torch.cuda.synchronize()
        got = hist.cpu().numpy().view(np.uint64)
        want, _ = oracle_hist(None, workloads.instance_rows(inst), per, D, B)
        assert np.array_equal(got, want)
        ntup = 4096 * (per // D)
        expect = ntup / B ** D
        chi2 = float(((got.astype(np.float64) - expect) ** 2).sum() / expect)
        dof = B ** D - 1
        assert abs(chi2 - dof) / np.sqrt(2 * dof) < 6, chi2
    finally:
        ph.phprng_destroy(ctx)


def test_serial_argument_errors(ph, torch):
    inst = workloads.draw_instances(4, seed=94)
    ctx = ph.phprng_create(32, inst, 0)
    wide = ph.phprng_create(64, workloads.draw_instances(2, width=64, seed=95), 0)
    try:
        h = torch.zeros(1 << 20, dtype=torch.int64, device="cuda")
        for D, B in [(0, 16), (9, 2), (1, 0), (2, 70000), (5, 32), (1, (1 << 20) + 1)]:
            with pytest.raises(ph.PhprngError):
                ph.phprng_serial_test(ctx, 0, 4, 100, D, B, h)
        with pytest.raises(ph.PhprngError):
            ph.phprng_serial_test(ctx, 0, 4, 100, 1, 16, np.zeros(16, dtype=np.uint64))   # host memory
        with pytest.raises(ph.PhprngError):
            ph.phprng_serial_test(wide, 0, 2, 100, 1, 16, h)                              # 64-bit moduli
        assert ph.phprng_get_state(ctx, 0)["pos"] == 0                                    # nothing ran
    finally:
        ph.phprng_destroy(ctx)
        ph.phprng_destroy(wide)


def test_poker_matches_oracle_and_probabilities(ph, torch):
    """Hands spanning lanes and warp groups over two ragged calls, equal to the
    oracle's counts; at scale the category frequencies match the exact
    probabilities (|z| < 6)."""
    inst = workloads.draw_instances(41, seed=96)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        rows = workloads.instance_rows(inst).copy()
        hist = torch.zeros(7, dtype=torch.int64, device="cuda")
        want = np.zeros(7, dtype=np.uint64)
        for per in (1003, 5000):
            ph.phprng_poker_test(ctx, 0, 41, per, hist)
            c, _, st, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
            for k in range(41):
                oracle.poker_hist(c[k], int(rows[k, 0]), want)
            rows[:, 4:6] = st
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
        s = ph.phprng_get_state(ctx, 40)
        assert (s["m"], s["s"], s["pos"]) == (int(rows[40, 4]), int(rows[40, 5]), 6003)
    finally:
        ph.phprng_destroy(ctx)
    inst = workloads.draw_instances(2048, seed=97)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        hist = torch.zeros(7, dtype=torch.int64, device="cuda")
        ph.phprng_poker_test(ctx, 0, 2048, 1 << 16, hist)
        h = hist.cpu().numpy().astype(np.float64)
        hands = 2048 * ((1 << 16) // 5)
        assert h.sum() == hands
        prob = np.array([0.3024, 0.504, 0.108, 0.072, 0.009, 0.0045, 0.0001])
        z = (h - hands * prob) / np.sqrt(hands * prob * (1 - prob))
        assert np.all(np.abs(z) < 6), z
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("lmax", [4, 32, 64])
def test_runs_match_oracle(ph, torch, lmax):
    """Runs spanning lanes, words and warp groups, carried across groups and
    left open at each call's end, over two ragged calls: equal to the oracle;
    the states continue."""
    inst = workloads.draw_instances(29, seed=98 + lmax)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        rows = workloads.instance_rows(inst).copy()
        hist = torch.zeros(2 * lmax, dtype=torch.int64, device="cuda")
        want = np.zeros(2 * lmax, dtype=np.uint64)
        for per in (257, 3000, 1):
            ph.phprng_runs_test(ctx, 0, 29, per, lmax, hist)
            c, _, st, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
            for k in range(29):
                oracle.runs_hist(c[k], int(rows[k, 0]), lmax, want)
            rows[:, 4:6] = st
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
        s = ph.phprng_get_state(ctx, 28)
        assert (s["m"], s["s"], s["pos"]) == (int(rows[28, 4]), int(rows[28, 5]), 3258)
    finally:
        ph.phprng_destroy(ctx)


def test_runs_small_modulus_long_runs(ph, torch):
    """A tiny modulus with a unit-like skip gives long runs (lengths above
    lmax land in the last bin) -- equal to the oracle."""
    from test_gpu_parity import primitive_root
    n, p = 1019, 509
    a = primitive_root(p)
    inst = {"n": [n, 1031], "e": [3, 7], "p": [p, p], "a": [a, a], "m0": [5, 900], "s0": [1, 2]}
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_ALLOW_SHARED_N)
    try:
        rows = np.array([[n, 3, p, a, 5, 1], [1031, 7, p, a, 900, 2]], dtype=np.uint64)
        hist = torch.zeros(2 * 8, dtype=torch.int64, device="cuda")
        ph.phprng_runs_test(ctx, 0, 2, 20000, 8, hist)
        c, _, _, _ = oracle.generate_many(rows, 20000, threads=2, want_r=False)
        want = np.zeros(16, dtype=np.uint64)
        for k in range(2):
            oracle.runs_hist(c[k], int(rows[k, 0]), 8, want)
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
    finally:
        ph.phprng_destroy(ctx)


@pytest.mark.parametrize("S,B,H", [(1 << 14, 1 << 20, 512), (256, 64, 300), (512, 1000, 64)])
def test_collisions_match_oracle(ph, torch, S, B, H):
    """Segments over two calls (a remainder of each call left out), counts equal
    to the oracle's; the streams continue."""
    inst = workloads.draw_instances(23, seed=120 + H)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        rows = workloads.instance_rows(inst).copy()
        hist = torch.zeros(H, dtype=torch.int64, device="cuda")
        want = np.zeros(H, dtype=np.uint64)
        total = 0
        for per in (3 * S + 1000, 2 * S):
            ph.phprng_collision_test(ctx, 0, 23, per, S, B, H, hist)
            c, _, st, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
            for k in range(23):
                oracle.collision_hist(c[k], int(rows[k, 0]), S, B, H, want)
            rows[:, 4:6] = st
            total += per
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
        s = ph.phprng_get_state(ctx, 22)
        assert (s["m"], s["s"], s["pos"]) == (int(rows[22, 4]), int(rows[22, 5]), total)
    finally:
        ph.phprng_destroy(ctx)


def test_collision_mean_at_scale(ph, torch):
    """4,096 streams x 2^16 numbers at the paper's sizes: the mean collision
    count of 16,384 segments within 5 standard errors of its expectation."""
    inst = workloads.draw_instances(4096, seed=125)
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        S, B, H = 1 << 14, 1 << 20, 512
        hist = torch.zeros(H, dtype=torch.int64, device="cuda")
        ph.phprng_collision_test(ctx, 0, 4096, 1 << 16, S, B, H, hist)
        h = hist.cpu().numpy().astype(np.float64)
        segs = 4096 * 4
        assert h.sum() == segs
        mean = float((h * np.arange(H)).sum()) / segs
        expect = S - B * (1 - (1 - 1 / B) ** S)
        assert abs(mean - expect) < 5 * np.sqrt(expect / segs), (mean, expect)
    finally:
        ph.phprng_destroy(ctx)


def test_collision_pieces_equal_separate_calls(ph, torch):
    """Calls larger than the kernel's 2^28-bin scratch run in pieces: along the
    streams (512 streams x 2^20 numbers, pieces of 2^19) and across them
    (20,000 streams x 2^14 + 300 numbers, slots in chunks of 16,384).  Each
    must give the histogram and the states of the same numbers taken in calls
    small enough for one piece (which the oracle tests check)."""
    S, B, H = 1 << 14, 1 << 20, 512
    for count, per, splits in ((512, 1 << 20, "len"), (20000, (1 << 14) + 300, "slots")):
        inst = workloads.draw_instances(count, seed=126 if splits == "len" else 127)
        one = ph.phprng_create(32, inst, 0)
        two = ph.phprng_create(32, inst, 0)
        try:
            h1 = torch.zeros(H, dtype=torch.int64, device="cuda")
            h2 = torch.zeros(H, dtype=torch.int64, device="cuda")
            ph.phprng_collision_test(one, 0, count, per, S, B, H, h1)
            if splits == "len":
                for _ in range(4):
                    ph.phprng_collision_test(two, 0, count, per // 4, S, B, H, h2)
            else:
                ph.phprng_collision_test(two, 0, 10000, per, S, B, H, h2)
                ph.phprng_collision_test(two, 10000, 10000, per, S, B, H, h2)
            torch.cuda.synchronize()
            assert int(h1.sum()) == count * (per // S)
            assert torch.equal(h1, h2)
            for i in (0, count // 2, count - 1):
                assert ph.phprng_get_state(one, i) == ph.phprng_get_state(two, i)
        finally:
            ph.phprng_destroy(one)
            ph.phprng_destroy(two)


def _interstream_oracle(rows, per, D, B):
    c, _, st, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
    return oracle.interstream_serial_hist(c, rows[:, 0], D, B), st


@pytest.mark.parametrize("Np,per,D,B,e", [(1, 1000, 2, 32, None), (3, 1001, 2, 16, None), (37, 777, 3, 10, None),
                                          (64, 513, 5, 4, None), (5, 2000, 1, 1 << 20, None),
                                          (1100, 40, 2, 1 << 10, None), (4, 9_000_001, 3, 16, 9),
                                          # D = 2, 4, 8 dividing Np: groups of D warps counting their
                                          # tuples as generated (ragged groups, long streams, shared
                                          # counters when B^D <= 224, group slots heaviest first, e = 9);
                                          # D = 1: the frequency test's kernel
                                          (64, 5003, 2, 32, None), (96, 2049, 4, 8, None),
                                          (128, 3001, 1, 1 << 16, None), (512, 70_001, 2, 1 << 10, None),
                                          (2048, 300, 2, 14, None), (64, 3001, 2, 4, None),
                                          (8, 5000, 2, 16, 9), (128, 1000, 4, 3, None),
                                          (1024, 300, 4, 4, None), (64, 2000, 8, 2, None),
                                          (2048, 257, 8, 3, None), (16, 3333, 8, 2, 17),
                                          # D = 3, 5, 6, 7 dividing Np: groups of 6, 5, 6, 7 warps per block
                                          (48, 1000, 3, 10, None), (30, 700, 5, 4, None),
                                          (30, 701, 5, 2, None), (36, 513, 6, 3, None),
                                          (21, 600, 7, 3, 9), (3 * 1024, 100, 3, 100, None)])
def test_interstream_matches_oracle(ph, torch, Np, per, D, B, e):
    """Interleaved order over Np streams: ragged tails (Np per mod D != 0),
    shared-memory and global counters, and 4 x 9,000,001 numbers at D = 3 in
    four chunks of about 2^25 numbers (a multiple of D per stream, so no
    tuple spans two chunks); two calls accumulate; the streams continue as
    after phprng_generate."""
    inst = workloads.draw_instances(Np, seed=500 + Np, exponent=e)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        rows = workloads.instance_rows(inst).copy()
        hist = torch.zeros(B ** D, dtype=torch.int64, device="cuda")
        want = np.zeros(B ** D, dtype=np.uint64)
        for call in range(2):
            ph.phprng_interstream_serial_test(ctx, 0, Np, per, D, B, hist)
            h, st = _interstream_oracle(rows, per, D, B)
            want += h
            rows[:, 4:6] = st
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
        s = ph.phprng_get_state(ctx, Np - 1)
        assert (s["m"], s["s"], s["pos"]) == (int(rows[-1, 4]), int(rows[-1, 5]), 2 * per)
    finally:
        ph.phprng_destroy(ctx)


def test_interstream_large_chunked_and_mixed_context(ph, torch):
    """A sub-range of 32-bit instances in a mixed-width context (ciphertexts
    kept as 64-bit words) over more than one chunk; 64-bit instances are
    rejected."""
    i32 = workloads.draw_instances(40, seed=511)
    i64 = workloads.draw_instances(3, width=64, seed=512)
    inst = workloads.concat_instances(i32, i64)
    ctx = ph.phprng_create(0, inst, 0)
    try:
        hist = torch.zeros(1 << 10, dtype=torch.int64, device="cuda")
        per = 900_001
        ph.phprng_interstream_serial_test(ctx, 1, 39, per, 2, 32, hist)
        want, _ = _interstream_oracle(workloads.instance_rows(i32)[1:], per, 2, 32)
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
        with pytest.raises(ph.PhprngError):
            ph.phprng_interstream_serial_test(ctx, 38, 3, 64, 2, 32, hist)
    finally:
        ph.phprng_destroy(ctx)


def test_interstream_paper_scale_chi_square(ph, torch):
    """32,768 streams (one of the paper's groupings) x 8,192 numbers with
    e = 9, pairs of the interleaved sequence into 2^20 bins: every tuple
    counted, chi-square unremarkable (|z| < 6)."""
    inst = workloads.draw_instances(32768, seed=513, exponent=9)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        hist = torch.zeros(1 << 20, dtype=torch.int64, device="cuda")
        ph.phprng_interstream_serial_test(ctx, 0, 32768, 8192, 2, 1 << 10, hist)
        torch.cuda.synchronize()
        got = hist.cpu().numpy().astype(np.float64)
        assert got.sum() == 32768 * 8192 // 2
        expect = got.sum() / got.size
        z = (((got - expect) ** 2).sum() / expect - (got.size - 1)) / (2 * (got.size - 1)) ** 0.5
        assert abs(z) < 6, z
    finally:
        ph.phprng_destroy(ctx)


# ------------------------------------------------------------ bins at exact multiples k/B
# floor(B R) is taken on the double R with one IEEE product; at an exact
# (c+1)/(n+1) = k/B that product can fall below k (B = 100: k = 29, 57, 58 on
# n = 2147483999, where n + 1 = 100 * 21474840).  The streams below are seeded
# so that such ciphertexts come out at chosen positions.
N100, P31, A31 = 2147483999, 2147483647, 784588716


def _is_prime(q):
    if q < 2:
        return False
    for d in (2, 3, 5, 7, 11, 13):
        if q % d == 0:
            return q == d
    d, r = q - 1, 0
    while d % 2 == 0:
        d, r = d // 2, r + 1
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


def _prime_with_divisor(B, start):
    n = start + (-1 - start) % B
    while not _is_prime(n):
        n += B
    return n


def _coprime_exponent(n, seed):
    rng = np.random.default_rng(seed)
    while True:
        e = int(rng.integers(3, n - 2))
        if np.gcd(e, n - 1) == 1:
            return e


def _seed_for(n, e, k, c, s0):
    """m0 such that number k (1-based) of the stream (n, e, P31, A31, m0, s0)
    is the ciphertext c: m_k = c^d (Eq. 2) = m0 + s_1 + .. + s_k (Eq. 6b)."""
    d = pow(e, -1, n - 1)
    ssum, s = 0, s0
    for _ in range(k):
        s = A31 * s % P31
        ssum += s
    return (pow(c, d, n) - ssum) % n


def _seed_pair(n, e, k, c_first, c_second):
    """(m0, s0) with number k equal to c_first and number k + 1 to c_second:
    the skip s_(k+1) must be the message difference, so it has to lie in
    [1, p-1]; returns None when it does not."""
    d = pow(e, -1, n - 1)
    delta = (pow(c_second, d, n) - pow(c_first, d, n)) % n
    if not 1 <= delta < P31:
        return None
    s0 = delta * pow(A31, -(k + 1), P31) % P31
    return _seed_for(n, e, k, c_first, s0), s0


def _exact_bins(c, n, B):
    return (B * (np.asarray(c, dtype=object) + 1)) // (n + 1)


def _exact_multiple_instances():
    """Streams on n = 2147483999 whose numbers at chosen positions (first
    number, inside a warp group, across a group boundary) are the three
    ciphertexts with a low double bin, for a straight-chain and a windowed
    exponent, plus ordinary streams."""
    rows = []
    targets = [(21474840 * k - 1) for k in (29, 57, 58)]
    for e in (3, _coprime_exponent(N100, 7)):
        for j, (k, c) in enumerate(zip((1, 77, 256), targets)):
            s0 = 1000 + 17 * j
            rows.append([N100, e, P31, A31, _seed_for(N100, e, k, c, s0), s0])
    rows = np.array(rows, dtype=np.uint64)
    extra = workloads.instance_rows(workloads.draw_instances(5, seed=4242))
    return np.concatenate([rows, extra])


def _ctx_from_rows(ph, rows):
    return ph.phprng_create(32, rows, ph.PHPRNG_ALLOW_SHARED_N)


@pytest.mark.parametrize("D", [1, 3])
def test_serial_bins_at_exact_multiples_match_oracle(ph, torch, D):
    """The paper's B = 100 (D = 3 is its three-dimensional serial test) on
    streams that emit the three low-double-bin ciphertexts: every counter
    equals the oracle's, which differs from exact-quotient binning."""
    rows = _exact_multiple_instances()
    per = 1000
    ctx = _ctx_from_rows(ph, rows)
    try:
        hist = torch.zeros(100 ** D, dtype=torch.int64, device="cuda")
        ph.phprng_serial_test(ctx, 0, len(rows), per, D, 100, hist)
        c, _, _, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
        want = np.zeros(100 ** D, dtype=np.uint64)
        for k in range(len(rows)):
            oracle.serial_hist(c[k], int(rows[k, 0]), D, 100, want)
        # the forced numbers are there, and exact binning would differ
        assert {int(x) for x in c[:6].ravel()} >= {21474840 * k - 1 for k in (29, 57, 58)}
        exact = np.zeros(100 ** D, dtype=np.uint64)
        for k in range(len(rows)):
            b = _exact_bins(c[k], int(rows[k, 0]), 100)
            nt = per // D
            idx = sum(b[d:nt * D:D] * 100 ** d for d in range(D))
            np.add.at(exact, np.array(idx, dtype=np.int64), 1)
        assert not np.array_equal(exact, want)
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
    finally:
        ph.phprng_destroy(ctx)


def test_interstream_bins_at_exact_multiples_match_oracle(ph, torch):
    """The interleaved order over the same streams from their seeds (so the
    forced ciphertexts come up in every case), single numbers and pairs into
    100 x 100 bins: all 11 streams (an odd count: the general form for pairs)
    and the first 10 (the fused pairs kernel)."""
    rows0 = _exact_multiple_instances()
    per = 600
    for D, Np in ((1, len(rows0)), (2, len(rows0)), (2, len(rows0) - 1)):
        rows = rows0[:Np]
        ctx = _ctx_from_rows(ph, rows)
        try:
            hist = torch.zeros(100 ** D, dtype=torch.int64, device="cuda")
            ph.phprng_interstream_serial_test(ctx, 0, Np, per, D, 100, hist)
            c, _, st, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
            want = oracle.interstream_serial_hist(c, rows[:, 0], D, 100)
            torch.cuda.synchronize()
            assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
            if D == 1:
                exact = np.zeros(100, dtype=np.uint64)
                for k in range(len(rows)):
                    np.add.at(exact, np.array(_exact_bins(c[k], int(rows[k, 0]), 100), dtype=np.int64), 1)
                assert not np.array_equal(exact, want)
            s = ph.phprng_get_state(ctx, Np - 1)
            assert (s["m"], s["s"], s["pos"]) == (int(st[-1, 0]), int(st[-1, 1]), per)
        finally:
            ph.phprng_destroy(ctx)


def test_collision_bins_at_exact_multiples_match_oracle(ph, torch):
    """Segments of 256 into B = 60000 bins (sparse, so a collision is rare):
    in each forced stream an earlier number of exact bin k - 1 is followed by
    the exact multiple k/B whose double product falls to bin k - 1 -- one
    collision that exact binning would not count."""
    B = 60000
    n = _prime_with_divisor(B, 3_000_000_000)
    t = (n + 1) // B
    low = [k for k in range(1, B) if (k / B) * B < k][:40]
    rows = []
    for e in (3, _coprime_exponent(n, 9)):
        for pos in (5, 130, 255):                   # the pair inside a group, across lanes, across groups
            for k in low:
                found = None
                for off in range(1, 2000):
                    found = _seed_pair(n, e, pos, (k - 1) * t + off, k * t - 1)
                    if found:
                        break
                if found:
                    rows.append([n, e, P31, A31, found[0], found[1]])
                    break
    assert len(rows) == 6
    rows = np.array(rows, dtype=np.uint64)
    S, H, per = 256, 8, 512
    ctx = _ctx_from_rows(ph, rows)
    try:
        hist = torch.zeros(H, dtype=torch.int64, device="cuda")
        ph.phprng_collision_test(ctx, 0, len(rows), per, S, B, H, hist)
        c, _, _, _ = oracle.generate_many(rows, per, threads=THREADS, want_r=False)
        want = np.zeros(H, dtype=np.uint64)
        exact = np.zeros(H, dtype=np.uint64)
        for k in range(len(rows)):
            oracle.collision_hist(c[k], n, S, B, H, want)
            b = _exact_bins(c[k], n, B)
            for g in range(0, per, S):
                seg = list(b[g:g + S])
                exact[min(S - len(set(seg)), H - 1)] += 1
        assert not np.array_equal(exact, want)
        torch.cuda.synchronize()
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
    finally:
        ph.phprng_destroy(ctx)
