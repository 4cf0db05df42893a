"""The fused-statistics call that allocates no GPU memory, for callers that
cannot allocate at the call site (a caching allocator owning the device's
memory, a latency-critical loop, allocation allowed only at start-up): its
results must equal those of the ordinary call, on two calls in a row.

This file is named to be collected last, so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1411_2484_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def test_no_alloc_statistics_equal_the_ordinary_call(ph, torch):
    inst = workloads.draw_instances(100, seed=701)
    ordinary = ph.phprng_create(32, inst, 0)
    fixed = ph.phprng_create(32, inst, 0)
    try:
        size = ph.STATS_DTYPE.itemsize
        for per in (1000, 777):                          # two calls in a row
            a = torch.zeros(100 * size, dtype=torch.uint8, device="cuda")
            b = torch.full((100 * size,), 255, dtype=torch.uint8, device="cuda")
            ph.phprng_generate(ordinary, 0, 100, per, None, None, a)
            ph.phprng_generate_stats_noalloc(fixed, 0, 100, per, b)
            torch.cuda.synchronize()
            sa = a.cpu().numpy().view(ph.STATS_DTYPE)
            sb = b.cpu().numpy().view(ph.STATS_DTYPE)
            assert sa.tobytes() == sb.tobytes()          # bit-exact, as every statistic is
            assert np.all(sb["count"] == per)
        for i in (0, 57, 99):
            assert ph.phprng_get_state(ordinary, i) == ph.phprng_get_state(fixed, i)
    finally:
        ph.phprng_destroy(ordinary)
        ph.phprng_destroy(fixed)


def test_no_alloc_rejects_sizes_beyond_its_scratch(ph, torch):
    inst = workloads.draw_instances(64, seed=702)
    ctx = ph.phprng_create(32, inst, 0)
    try:
        out = torch.empty(64 * ph.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        with pytest.raises(ph.PhprngError) as ei:
            ph.phprng_generate_stats_noalloc(ctx, 0, 64, 1 << 17, out)   # 2*8*2^17 > 2^20
        assert ei.value.status == ph.PHPRNG_EINVAL and "2^20" in str(ei.value)
        assert ph.phprng_get_state(ctx, 0)["pos"] == 0   # nothing ran
    finally:
        ph.phprng_destroy(ctx)
