"""GPU tests of the Fourier test (Tests section) through the C ABI: the
coefficients must equal the oracle's (numpy's FFT of the oracle's R) within
FP64 transform rounding, the histogram must be exactly the binning of the
library's own coefficients and differ from the oracle's only for parts within
rounding of a bin edge, and the streams must continue as after
phprng_generate."""
import os

import numpy as np
import pytest

import oracle
from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
# |FFT error| for M <= 2^20 points of |x| <= 1/2: about eps log2(M) sqrt(M) / sqrt(M)
# times a small constant; 1e-12 leaves three orders of margin and still catches
# any wrong twiddle, index or scale (those move coefficients by ~0.1).
ATOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def _run(ph, torch, inst, per, lgM, nbins, w, calls=1, want_coef=True):
    """Library histogram and coefficients over `calls` consecutive calls."""
    count = len(inst["n"])
    M = 1 << lgM
    ctx = ph.phprng_create(32, inst, 0)
    try:
        hist = torch.zeros(nbins, dtype=torch.int64, device="cuda")
        coefs = []
        for _ in range(calls):
            coef = torch.empty(count * per, dtype=torch.float64, device="cuda") if want_coef else None
            ph.phprng_fourier_test(ctx, 0, count, per, lgM, nbins, w, hist, coef)
            if want_coef:
                coefs.append(coef.cpu().numpy().view(np.complex128).reshape(count, per // M, M // 2))
        torch.cuda.synchronize()
        states = [ph.phprng_get_state(ctx, i) for i in range(count)]
    finally:
        ph.phprng_destroy(ctx)
    return hist.cpu().numpy().view(np.uint64), coefs, states


def _oracle(inst, per, lgM, calls=1):
    """Oracle coefficients [calls][count, seqs, M/2] and final states."""
    rows = workloads.instance_rows(inst).copy()
    out = []
    for _ in range(calls):
        _, r, st, _ = oracle.generate_many(rows, per, threads=THREADS, want_c=False)
        out.append(np.stack([oracle.fourier_coefficients(r[k], 1 << lgM) for k in range(len(rows))]))
        rows[:, 4:6] = st
    return out, rows


def _check_hist(hist, gpu_coefs, want_coefs, nbins, w):
    """hist is exactly the binning of the library's coefficients, and those
    bins differ from the oracle's only where the oracle's part lies within
    rounding of a bin edge."""
    mine = np.zeros(nbins, dtype=np.uint64)
    for c in gpu_coefs:
        oracle.fourier_hist(c, nbins, w, mine)
    assert np.array_equal(hist, mine)
    g = np.concatenate([c.reshape(-1) for c in gpu_coefs])
    o = np.concatenate([c.reshape(-1) for c in want_coefs])
    for gp, op in ((g.real, o.real), (g.imag, o.imag)):
        diff = oracle.fourier_bin(gp, nbins, w) != oracle.fourier_bin(op, nbins, w)
        if diff.any():
            scaled = (op[diff] + w) * (nbins / (2.0 * w))
            assert np.all(np.abs(scaled - np.round(scaled)) < 1e-9)


@pytest.mark.parametrize("lgM,per", [(2, 4 * 7), (3, 8 * 5), (5, 32 * 3), (10, 1024 * 3),
                                     (11, 2048 * 2), (16, 1 << 17)])
def test_fourier_matches_oracle(ph, torch, lgM, per):
    """Odd and even log2 M (square and 2:1 four-step splits), two consecutive
    calls, 11 instances with drawn exponents."""
    inst = workloads.draw_instances(11, seed=300 + lgM)
    nbins, w = 97, 1.25
    hist, gpu, states = _run(ph, torch, inst, per, lgM, nbins, w, calls=2)
    want, rows = _oracle(inst, per, lgM, calls=2)
    for g, o in zip(gpu, want):
        assert g.shape == o.shape
        assert np.max(np.abs(g - o)) < ATOL
    _check_hist(hist, gpu, want, nbins, w)
    for i in (0, 5, 10):
        assert (states[i]["m"], states[i]["s"], states[i]["pos"]) == \
            (int(rows[i, 4]), int(rows[i, 5]), 2 * per)


def test_fourier_largest_M_and_global_histogram(ph, torch):
    """M = 2^20 (the largest transform, 1024 x 1024) and 4,096 bins (above the
    shared-memory histogram limit, so counters go straight to global memory)."""
    inst = workloads.draw_instances(3, seed=320, exponent=9)
    lgM, per = 20, 2 << 20
    hist, gpu, _ = _run(ph, torch, inst, per, lgM, 4096, 1.5)
    want, _ = _oracle(inst, per, lgM)
    assert np.max(np.abs(gpu[0] - want[0])) < ATOL
    _check_hist(hist, gpu, want, 4096, 1.5)


def test_fourier_batches(ph, torch):
    """72 instances x 2^20 numbers: more than one 2^26-number batch of R, so the
    second batch's coefficients land at the right offsets of coef_out."""
    inst = workloads.draw_instances(72, seed=321, exponent=9)
    lgM, per = 12, 1 << 20
    hist, gpu, _ = _run(ph, torch, inst, per, lgM, 64, 1.0)
    want, _ = _oracle(inst, per, lgM)
    assert np.max(np.abs(gpu[0] - want[0])) < ATOL
    _check_hist(hist, gpu, want, 64, 1.0)


def test_fourier_variance_at_scale(ph, torch):
    """4,096 streams x 2^16 numbers, M = 2^16: the pooled parts have mean 0 and
    variance 1/24 (k = 0 contributes 1/12 real and 0 imaginary; every other
    coefficient 1/24 in each part), from the histogram's bin centres."""
    inst = workloads.draw_instances(4096, seed=322)
    nbins, w = 8192, 2.0
    hist, _, _ = _run(ph, torch, inst, 1 << 16, 16, nbins, w, want_coef=False)
    h = hist.astype(np.float64)
    assert h.sum() == 2 * 4096 * (1 << 15)
    assert h[0] == 0 and h[-1] == 0                    # nothing beyond 11 standard deviations
    centre = -w + (np.arange(nbins) + 0.5) * (2 * w / nbins)
    mean = (h * centre).sum() / h.sum()
    var = (h * centre ** 2).sum() / h.sum() - mean ** 2
    se = np.sqrt(2.0 / h.sum())                        # relative standard error of a variance
    assert abs(mean) < 6 * np.sqrt(1 / 24 / h.sum())
    assert abs(var * 24 - 1) < 6 * se + 1e-4           # 1e-4: binning (Sheppard) bias bound


def test_fourier_argument_errors(ph, torch):
    inst = workloads.draw_instances(2, seed=323)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        hist = torch.zeros(16, dtype=torch.int64, device="cuda")
        for args in ((1, 16, 1.0, 8), (21, 16, 1.0, 1 << 21), (4, 16, 1.0, 24), (4, 0, 1.0, 32),
                     (4, 16, 0.0, 32), (4, 16, -1.0, 32)):
            lgM, nb, w, per = args
            with pytest.raises(RuntimeError):
                ph.phprng_fourier_test(ctx, 0, 2, per, lgM, nb, w, hist)
        with pytest.raises(RuntimeError):
            ph.phprng_fourier_test(ctx, 0, 2, 32, 4, 16, 1.0, torch.zeros(16, dtype=torch.int64))
        with pytest.raises(RuntimeError):
            ph.phprng_fourier_test(ctx, 1, 2, 32, 4, 16, 1.0, hist)
        assert ph.phprng_get_state(ctx, 0)["pos"] == 0
    finally:
        ph.phprng_destroy(ctx)
    wide = workloads.draw_instances(1, width=64, seed=324)
    ctx = ph.phprng_create(64, wide, 0)
    try:
        with pytest.raises(RuntimeError):
            ph.phprng_fourier_test(ctx, 0, 1, 32, 4, 16, 1.0, hist)
    finally:
        ph.phprng_destroy(ctx)


def test_fourier_bench_size_sampled(ph, torch):
    """The benchmark's launch: the first 256 instances of the plain 32-bit
    workload x 2^20 numbers at M = 2^20, 8,192 bins over [-2, 2).  Sampled
    sequences (first, middle, last instance, the last in the fourth 2^26-number
    batch) equal the oracle's; the histogram holds every part and is the
    binning of all the library's coefficients."""
    inst = workloads.workload_instances("plain32_65536x4096x64", 256)
    N, per, lgM, nbins, w = 256, 1 << 20, 20, 8192, 2.0
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    try:
        hist = torch.zeros(nbins, dtype=torch.int64, device="cuda")
        coef = torch.empty(N * per, dtype=torch.float64, device="cuda")
        ph.phprng_fourier_test(ctx, 0, N, per, lgM, nbins, w, hist, coef)
        torch.cuda.synchronize()
        h = hist.cpu().numpy().view(np.uint64)
        assert int(h.sum()) == N * per
        X = coef.cpu().numpy().view(np.complex128).reshape(N, per // 2)
        mine = oracle.fourier_hist(X, nbins, w)
        assert np.array_equal(h, mine)
    finally:
        ph.phprng_destroy(ctx)
    rows = workloads.instance_rows(inst)
    for i in (0, 127, 200, 255):
        _, r, _, _ = oracle.generate_many(rows[i:i + 1], per, threads=1, want_c=False)
        want = oracle.fourier_coefficients(r[0], 1 << lgM)[0]
        assert np.max(np.abs(X[i] - want)) < ATOL, i
