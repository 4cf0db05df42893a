"""GPU tests of the full-period pattern enumeration (phprng_pattern) through the
C ABI: equal to the oracle's enumeration (itself pinned against brute-force
counts over whole periods), and the paper's instance at scale."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def run(ph, torch, n, e, p, a, c_lo, L0, D, nb):
    hist = torch.zeros(nb ** (D - 1), dtype=torch.int64, device="cuda")
    ph.phprng_pattern(n, e, p, a, c_lo, L0, D, nb, hist)
    torch.cuda.synchronize()
    return hist.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("n,p,e", [(1019, 509, 3), (1031, 103, 7), (4294967087, 65537, 9),
                                   (4294967087, 65537, 4294967085)])
@pytest.mark.parametrize("D,nb", [(2, 8), (3, 16), (5, 4)])
def test_pattern_matches_oracle(ph, torch, n, p, e, D, nb):
    from test_gpu_parity import primitive_root
    a = primitive_root(p)
    c_lo, L0 = (0, n) if n < 5000 else (123456, 24)
    got = run(ph, torch, n, e, p, a, c_lo, L0, D, nb)
    want = oracle.pattern_hist(n, e, p, a, c_lo, L0, D, nb)
    assert np.array_equal(got, want)


def test_pattern_paper_instance_uniform(ph, torch):
    """The instance of the paper's pattern figures (n = 4294967087, p = 2^31-1,
    a = 784588716, e = 9): L0 (p-1) points, and over 4,096 volumes of a
    three-dimensional pattern a chi-square consistent with uniform (|z| < 6)."""
    n, p, a, e = 4294967087, 2147483647, 784588716, 9
    D, nb, L0 = 3, 64, 2
    got = run(ph, torch, n, e, p, a, 1000, L0, D, nb).astype(np.float64)
    assert got.sum() == L0 * (p - 1)
    L1 = -(-n // nb)
    widths = np.array([min(L1, n - b * L1) for b in range(nb)], dtype=np.float64) / n
    expect = L0 * (p - 1) * np.outer(widths, widths).reshape(-1)    # index b1 + nb b2
    chi2 = float(((got - expect) ** 2 / expect).sum())
    dof = nb ** (D - 1) - 1
    assert abs(chi2 - dof) / np.sqrt(2 * dof) < 6, chi2


def test_pattern_argument_errors(ph, torch):
    h = torch.zeros(1 << 10, dtype=torch.int64, device="cuda")
    n, p, a = 1019, 509, 2
    for args in [(n, 3, p, a, 0, 0, 2, 8), (n, 3, p, a, 1000, 20, 2, 8), (n, 3, p, a, 0, 8, 1, 8),
                 (n, 3, p, a, 0, 8, 9, 2), (n, 3, p, a, 0, 8, 3, 5000), (n, 4, p, a, 0, 8, 2, 8),
                 (1021, 3, p, a, 0, 8, 2, 8)]:
        with pytest.raises(ph.PhprngError):
            ph.phprng_pattern(*args, h)
    with pytest.raises(ph.PhprngError):
        ph.phprng_pattern(n, 3, p, a, 0, 8, 2, 8, np.zeros(8, dtype=np.uint64))   # host memory


@pytest.mark.parametrize("n,e", [(1019, 3), (4099, 5), (4294967087, 9), (4294967087, 4294967085)])
@pytest.mark.parametrize("b", [1, 12345])
@pytest.mark.parametrize("D,nb", [(2, 8), (3, 16), (4, 4)])
def test_pattern_const_matches_oracle(ph, torch, n, e, b, D, nb):
    """The constant-skip (b = 1: unit skip) full-period pattern equals the
    oracle's (itself pinned against brute force over whole periods)."""
    b = b % n or 1
    c_lo, L0 = (0, n) if n < 5000 else (77, 100000)
    hist = torch.zeros(nb ** (D - 1), dtype=torch.int64, device="cuda")
    ph.phprng_pattern_const(n, e, b, c_lo, L0, D, nb, hist)
    torch.cuda.synchronize()
    want = oracle.pattern_const_hist(n, e, b, c_lo, L0, D, nb)
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)


def test_pattern_const_whole_period_unit_skip(ph, torch):
    """The unit skip over a whole 32-bit period (the paper's Fig. 2 generator,
    n = 4294967087, e = 9): n points, and with D = 2 every column of the
    pattern holds exactly as many points as values of c1 fall in it."""
    n, e = 4294967087, 9
    nb = 256
    hist = torch.zeros(nb, dtype=torch.int64, device="cuda")
    ph.phprng_pattern_const(n, e, 1, 0, n, 2, nb, hist)
    h = hist.cpu().numpy().view(np.uint64)
    L1 = -(-n // nb)
    want = np.array([min(L1, n - k * L1) for k in range(nb)], dtype=np.uint64)
    assert np.array_equal(h, want)


@pytest.mark.parametrize("n,p,e,D,nb,L1", [(1019, 509, 3, 2, 8, 37), (1031, 103, 7, 3, 5, 100),
                                           (1019, 509, 3, 2, 64, 1), (1019, 509, 3, 3, 8, 1),
                                           (4294967087, 65537, 9, 2, 64, 1 << 20),
                                           (4294967087, 65537, 9, 3, 4, 1 << 28)])
def test_pattern_region_matches_oracle(ph, torch, n, p, e, D, nb, L1):
    """Regions of cells of width L1 (tuples with a successor at or above
    nb L1 left out), pseudorandom and unit skip, against the oracle."""
    from test_gpu_parity import primitive_root
    a = primitive_root(p)
    c_lo, L0 = (0, n) if n < 5000 else (77, 24)
    hist = torch.zeros(nb ** (D - 1), dtype=torch.int64, device="cuda")
    ph.phprng_pattern_region(n, e, p, a, c_lo, L0, D, nb, L1, hist)
    torch.cuda.synchronize()
    assert np.array_equal(hist.cpu().numpy().view(np.uint64),
                          oracle.pattern_region_hist(n, e, p, a, c_lo, L0, D, nb, L1))
    hist.zero_()
    L0c = min(L0 * 50, n - c_lo)
    ph.phprng_pattern_const_region(n, e, 1, c_lo, L0c, D, nb, L1, hist)
    torch.cuda.synchronize()
    assert np.array_equal(hist.cpu().numpy().view(np.uint64),
                          oracle.pattern_const_region_hist(n, e, 1, c_lo, L0c, D, nb, L1))
    with pytest.raises(ph.PhprngError):
        ph.phprng_pattern_region(n, e, p, a, c_lo, L0, D, nb, 0, hist)


def test_pattern_region_paper_figures(ph, torch):
    """The paper's figure regions: Fig. 2's 16 cells of (2^18)^2 for the unit
    skip with n = 2^32 - 5, e = 9 equal the oracle's; Fig. 3's 2^7 x 2^7
    square (pseudorandom skip, n = 4294967087, p = 2^31 - 1, e = 9): every
    pair at most once, none on the diagonal, about half the pairs present;
    Fig. 4's 2^9 x 2^16 x 2^16 slab in 16 subslabs, each near 16."""
    n2 = 4294967291
    h = torch.zeros(4, dtype=torch.int64, device="cuda")
    for i in range(4):
        h.zero_()
        ph.phprng_pattern_const_region(n2, 9, 1, i << 18, 1 << 18, 2, 4, 1 << 18, h)
        torch.cuda.synchronize()
        assert np.array_equal(h.cpu().numpy().view(np.uint64),
                              oracle.pattern_const_region_hist(n2, 9, 1, i << 18, 1 << 18, 2, 4, 1 << 18))
    n, p, a, e = 4294967087, 2147483647, 784588716, 9
    sq = np.zeros((128, 128), dtype=np.int64)
    row = torch.zeros(128, dtype=torch.int64, device="cuda")
    for c0 in range(128):
        row.zero_()
        ph.phprng_pattern_region(n, e, p, a, c0, 1, 2, 128, 1, row)
        torch.cuda.synchronize()
        sq[c0] = row.cpu().numpy()
    assert sq.max() <= 1 and np.trace(sq) == 0
    rho = (p - 1) / n                                   # about 0.5
    assert abs(sq.sum() - rho * 128 * 128) < 6 * (rho * (1 - rho) * 128 * 128) ** 0.5
    slab = torch.zeros(16, dtype=torch.int64, device="cuda")
    ph.phprng_pattern_region(n, e, p, a, 0, 1 << 9, 3, 4, 1 << 14, slab)
    torch.cuda.synchronize()
    cells = slab.cpu().numpy()
    assert cells.sum() > 0 and abs(cells.mean() - 16) < 6 * 4 / 4 and cells.max() < 16 + 6 * 4


def test_pattern_region_three_dimensional_slab_matches_oracle(ph, torch):
    """Fig. 4's construction (D = 3, c0 in [0, 2^9), the paper's instance
    n = 4294967087, e = 9) with a skip generator small enough for the oracle
    (p = 65537, a = 3) and cells of 2^22, so that about 500 points fall in the
    4 x 4 subslabs: every counter equals the oracle's (the region limit and the
    cell width of the slab call, checked exactly)."""
    n, e, p, a = 4294967087, 9, 65537, 3
    hist = torch.zeros(16, dtype=torch.int64, device="cuda")
    ph.phprng_pattern_region(n, e, p, a, 0, 1 << 9, 3, 4, 1 << 22, hist)
    torch.cuda.synchronize()
    want = oracle.pattern_region_hist(n, e, p, a, 0, 1 << 9, 3, 4, 1 << 22)
    assert want.sum() > 300
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), want)
