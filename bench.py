#!/usr/bin/env python
"""Benchmark of the plain 32-bit generator at scale.

Workload (one step = one generate call): 65,536 independent instances (32-bit
safe primes, random exponents e in [3, n-2] coprime to n-1, seeded), 4,096
numbers each per call, R_k in FP64 written to HBM (2 GiB per call); the
instances advance through consecutive calls via their stored state, as in the
64-call run.  Metric: pseudorandom numbers per second, bit-exact with the CPU
oracle (tests/test_gpu_parity.py checks this launch at full size).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank owns its own 65,536
instances (weak scaling, no data-path collective); the timed region is
bracketed by barriers and the slowest rank's time is reported.
--impl reference times the CPU oracle on the host cores instead (rank 0).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "plain32_65536x4096x64"
METRIC = "PRNs/s on 1 GB300 bit-exact vs oracle, % of IMAD/HBM roofline; p99 serve latency"
# Roofline of the 32-bit path: the integer multiplier.  A GB300 SM issues 64
# 32-bit integer multiplies (IMAD, one 32-bit product half each) per clock
# (CUDA C++ Programming Guide, arithmetic throughput table); 152 SMs at the
# 2,070 MHz maximum SM clock.
SMS, MULS_PER_CLK_SM, SM_MAX_MHZ = 152, 64, 2070.0
PEAK_TMULS = SMS * MULS_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--modes", default="fused,serial,interstream,consumers,small_e,pattern,fourier,figures,wide64,c0,batched,served",
                    help="comma-separated extra measurements after the headline, or 'none'")
    return ap.parse_args()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def algorithmic_muls(e_values, per_inst):
    """32-bit multiply halves per call: 4 per modular product (a 32x32 product
    is two halves, the reduction one low and one high half), with
    (bitlen(e)-1) squarings + (popcount(e)-1) multiplications per Eq. 9c and
    one product for the skip update Eq. 9a."""
    total = 0
    for e in e_values:
        e = int(e)
        total += 4 * ((e.bit_length() - 1) + (bin(e).count("1") - 1) + 1)
    return total * per_inst


class ClockSampler:
    """nvidia-smi samples every 20 ms, started before the warm-up so that its
    own start-up is over when the timed region begins; stop(t0, t1) keeps the
    samples whose timestamps fall inside the timed wall-clock window [t0, t1]
    (the nearest ones when the window is shorter than the sampling period)."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid, period_ms=20):
        self.proc = None
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                   "-lms", str(period_ms)]
            if uuid:
                cmd += ["-i", uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    @staticmethod
    def _when(stamp):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((self._when(f[0]), float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if r[0] is not None and t0 is not None and t0 <= r[0] <= t1]
        note = "samples inside the timed window"
        if not inside and t0 is not None:
            timed_rows = [r for r in rows if r[0] is not None]
            if timed_rows:
                mid = 0.5 * (t0 + t1)
                timed_rows.sort(key=lambda r: abs(r[0] - mid))
                inside = timed_rows[:2]
                note = "window shorter than the sampling period: the two samples nearest to it"
        if not inside:
            inside, note = rows, "all samples (no timestamps)"
        reasons = set()
        for r in inside:
            for nm, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside),
                "samples": len(inside), "samples_total": len(rows), "note": note,
                "reasons": sorted(reasons)}


def profile_entry(kernel):
    """The committed ncu record of a kernel (DRAM bytes per launch, pipe
    instruction counts per number), if it was taken on the current kernel
    source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))[kernel]
    except (KeyError, ValueError):
        return None
    h = hashlib.sha256()
    for f in d.get("sources", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != d.get("sha256"):
        return None
    return d


def profile_traffic(kernel):
    d = profile_entry(kernel)
    return d.get("bytes_per_launch") if d else None


def cpu_baseline(inst, per_inst, target_s=12.0):
    """The oracle as it stands on this host's cores, on a bounded sample."""
    import oracle
    from paper_1411_2484_gb300 import workloads
    rows = workloads.instance_rows(inst)
    cores = host_cores()
    probe = min(len(rows), max(cores, 32))
    t0 = time.perf_counter()
    oracle.generate_many(rows[:probe], per_inst, threads=cores, want_c=False)
    dt0 = time.perf_counter() - t0
    count = int(min(len(rows), max(probe, probe * target_s / max(dt0, 1e-3))))
    t0 = time.perf_counter()
    oracle.generate_many(rows[:count], per_inst, threads=cores, want_c=False)
    dt = time.perf_counter() - t0
    # one core on a smaller sample (about 2 s)
    one = max(1, min(len(rows), int(2.0 * count / max(dt, 1e-3) / max(cores, 1))))
    t0 = time.perf_counter()
    oracle.generate_many(rows[:one], per_inst, threads=1, want_c=False)
    dt1 = time.perf_counter() - t0
    return {"value": count * per_inst / dt, "unit": "PRNs/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of the %d instances x %d numbers (R stored), %.1f s"
                      % (count, len(rows), per_inst, dt),
            "value_1core": one * per_inst / dt1, "sample_1core": "first %d instances, %.1f s" % (one, dt1),
            "cpu_model": cpu_model()}


def cpu_model():
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def muls_per_number(e, wide):
    """32-bit product halves per number (the algorithmic count of the roofline): the
    binary method's squarings and multiplications of Eq. 9c plus the skip
    product of Eq. 9a; 4 halves per 32-bit Montgomery product, 20 per 64-bit
    one (full 128-bit product 8, low word of q 4, high word of q n 8)."""
    e = int(e)
    mulmods = (e.bit_length() - 1) + (bin(e).count("1") - 1)
    return 20 * mulmods + 4 if wide else 4 * (mulmods + 1)


def timed(torch, stream, fn, steps, warmup=2):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def mode_fused(ph, torch, ctx, N, per, stream, steps):
    """The same workload in fused mode: per-stream statistics, no R stores."""
    sb = torch.empty(N * ph.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_generate(ctx, 0, N, per, None, None, sb, stream),
               steps)
    return {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
            "workload": "plain32 65,536 x 4,096, statistics only (72 MB/call)"}


def mode_small_e(ph, torch, stream, peak):
    """The plain 32-bit scale with e = 9 for every instance (the paper's
    recommended exponent): R to HBM, 2 GiB per call.  Few products per number,
    so the roofline is the lower of the multiplier and the HBM write bound."""
    from paper_1411_2484_gb300 import workloads
    inst = workloads.workload_instances("plain32_e9_65536x4096")
    N, per = 65536, 4096
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
    try:
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        ms = timed(torch, stream, lambda: ph.phprng_generate(ctx, 0, N, per, None, r, None, stream),
                   16, warmup=3)
    finally:
        ph.phprng_destroy(ctx)
    prn_s = N * per / ms * 1e3
    mul_bound = peak * 1e12 / muls_per_number(9, False)
    hbm = measured_hbm_gbs()
    hbm_bound = (hbm or 0) * 1e9 / 8
    if hbm and hbm_bound < mul_bound:
        roof = {"bound": "hbm", "achieved": prn_s * 8 / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": prn_s * 8 / 1e9 / hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    else:
        roof = {"bound": "alu", "achieved": prn_s * muls_per_number(9, False) / 1e12, "peak": peak,
                "unit": "T mul32/s", "frac": prn_s / mul_bound}
    return {"value": prn_s, "unit": "PRNs/s", "ms_per_call": ms,
            "workload": "65,536 safe 32-bit primes, e = 9, x 4,096 numbers per call (R, 2 GiB)",
            "roofline": roof}


def mode_c0(ph, torch, stream, peak):
    """The 4-instance reference workload (4 safe 32-bit primes, random
    exponents, 2^20 numbers each, c and R stored): four warps' worth of
    instances, so the call runs as a split launch (every stream cut into
    chunks after a skip-sum pre-pass, Eq. 6 over chunks)."""
    from paper_1411_2484_gb300 import workloads
    name = "pr1_ref_32bit_4x2^20"
    w = workloads.WORKLOADS[name]
    inst = workloads.workload_instances(name)
    N, per = w["instances"], w["per_inst"]
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
    try:
        c = torch.empty(N * per, dtype=torch.int32, device="cuda")
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        ms = timed(torch, stream, lambda: ph.phprng_generate(ctx, 0, N, per, c, r, None, stream),
                   20, warmup=3)
    finally:
        ph.phprng_destroy(ctx)
    prn_s = N * per / ms * 1e3
    muls = algorithmic_muls(inst["e"], per)
    achieved = muls / (ms * 1e-3) / 1e12
    return {"value": prn_s, "unit": "PRNs/s", "ms_per_call": ms,
            "workload": "%s: 4 x 2^20 numbers per call, c (uint32) and R (FP64) stored, "
                        "split launch (chunk pre-pass + generator)" % name,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T mul32/s",
                         "frac": achieved / peak, "algorithmic_muls_per_call": muls,
                         "peak_source": "152 SMs x 64 IMAD/clk x 2070 MHz (unit counts x max clock)"}}


def mode_serial(ph, torch, ctx, N, per, stream):
    """The two-dimensional serial test of the Tests section (pairs into 2^20
    bins) fused on the plain workload: nothing but the histogram is written."""
    D, B = 2, 1 << 10
    hist = torch.zeros(B ** D, dtype=torch.int64, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_serial_test(ctx, 0, N, per, D, B, hist, stream), 8)
    torch.cuda.synchronize()
    got = hist.cpu().numpy().astype(np.float64)
    expect = got.sum() / B ** D
    chi2 = float(((got - expect) ** 2).sum() / expect)
    dof = B ** D - 1
    return {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
            "workload": "plain32 65,536 x 4,096, pairs into 2^20 bins (8 MiB histogram)",
            "chi2_z": (chi2 - dof) / (2 * dof) ** 0.5}


def mode_pattern(ph, torch, stream, L0=128):
    """The full-period three-dimensional pattern of the paper's instance
    (n = 4294967087, p = 2^31-1, a = 784588716, e = 9) in 2^24 volumes of
    L0 L1^2, L0 = 2^7, by the O(p L0) enumeration: L0 (p-1) points, two
    exponentiations each; chi-square of the volumes against uniform."""
    n, p, a, e, D, nb = 4294967087, 2147483647, 784588716, 9, 3, 4096
    hist = torch.zeros(nb ** (D - 1), dtype=torch.int64, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_pattern(n, e, p, a, 0, L0, D, nb, hist, stream), 1,
               warmup=0)
    got = hist.cpu().numpy().astype(np.float64)
    L1 = -(-n // nb)
    widths = np.array([min(L1, n - b * L1) for b in range(nb)], dtype=np.float64) / n
    expect = L0 * (p - 1) * np.outer(widths, widths).reshape(-1)
    chi2 = float(((got - expect) ** 2 / expect).sum())
    dof = nb ** (D - 1) - 1
    points = L0 * (p - 1)
    return {"value": points / ms * 1e3, "unit": "points/s", "ms": ms,
            "exponentiations_per_s": 2 * points / ms * 1e3,
            "workload": "paper's pattern instance, D = 3, L0 = 2^7, 2^24 volumes (2^38 points)",
            "chi2_z": (chi2 - dof) / (2 * dof) ** 0.5}


def mode_figures(ph, torch, stream):
    """The settings of the paper's pattern figures as tables, from the
    full-period region calls: Fig. 2 (unit skip, n = 2^32 - 5, e = 9; 16 cells
    of (2^18)^2 near the origin), Fig. 3 (pseudorandom skip, n = 4294967087,
    p = 2^31 - 1, a = 784588716, e = 9; the 2^7 x 2^7 square: pairs present,
    most in one cell, on the diagonal) and Fig. 4 (the same instance; the
    2^9 x 2^16 x 2^16 slab in 16 subslabs)."""
    t0 = time.perf_counter()
    fig2 = []
    h = torch.zeros(4, dtype=torch.int64, device="cuda")
    for i in range(4):
        h.zero_()
        ph.phprng_pattern_const_region(4294967291, 9, 1, i << 18, 1 << 18, 2, 4, 1 << 18, h, stream)
        torch.cuda.synchronize()
        fig2.append([int(v) for v in h.cpu().numpy()])
    n, p, a, e = 4294967087, 2147483647, 784588716, 9
    sq = torch.zeros((128, 128), dtype=torch.int64, device="cuda")
    for c0 in range(128):
        ph.phprng_pattern_region(n, e, p, a, c0, 1, 2, 128, 1, sq[c0], stream)
    torch.cuda.synchronize()
    sqn = sq.cpu().numpy()
    slab = torch.zeros(16, dtype=torch.int64, device="cuda")
    ph.phprng_pattern_region(n, e, p, a, 0, 1 << 9, 3, 4, 1 << 14, slab, stream)
    torch.cuda.synchronize()
    fig4 = slab.cpu().numpy().reshape(4, 4)
    return {"seconds": time.perf_counter() - t0,
            "fig2_cells_ck_rows_ck1_cols": fig2,
            "fig3_pairs_present": int(sqn.sum()), "fig3_max_per_pair": int(sqn.max()),
            "fig3_on_diagonal": int(np.trace(sqn)), "fig3_expected": 128 * 128 * (p - 1) / n,
            "fig4_subslabs_ck1_rows_ck2_cols": [[int(v) for v in r] for r in fig4.T],
            "fig4_expected_per_cell": (1 << 41) / 16 * (p - 1) / n ** 2}


def mode_interstream(ph, torch, ctx, N, per, stream):
    """The paper's interstream ordering (number 1 of every stream, then
    number 2 of every stream, ...) over the plain workload's 65,536 streams,
    pairs of that sequence into 2^20 bins."""
    D, B = 2, 1 << 10
    hist = torch.zeros(B ** D, dtype=torch.int64, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_interstream_serial_test(ctx, 0, N, per, D, B, hist, stream), 4)
    torch.cuda.synchronize()
    got = hist.cpu().numpy().astype(np.float64)
    expect = got.sum() / B ** D
    chi2 = float(((got - expect) ** 2).sum() / expect)
    dof = B ** D - 1
    return {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
            "workload": "plain32 65,536 streams x 4,096, interleaved order, pairs into 2^20 bins",
            "chi2_z": (chi2 - dof) / (2 * dof) ** 0.5}


def mode_consumers(ph, torch, ctx, N, per, stream):
    """The poker, runs and collision tests of the Tests section, each fused on
    the generator over 2^28 numbers: poker on the plain workload's 65,536 x
    4,096 (hands of five numbers, ten denominations), runs on the same streams
    (lengths to 32), collision on 16,384 of its instances x 16,384 numbers (the
    paper's segments of 2^14 numbers into 2^20 bins).  Only the counters are
    written."""
    out = {}
    hist = torch.zeros(7, dtype=torch.int64, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_poker_test(ctx, 0, N, per, hist, stream), 4)
    out["poker"] = {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
                    "workload": "plain32 65,536 x 4,096, hands of five into 7 categories"}
    lmax = 32
    hist = torch.zeros(2 * lmax, dtype=torch.int64, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_runs_test(ctx, 0, N, per, lmax, hist, stream), 4)
    out["runs"] = {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
                   "workload": "plain32 65,536 x 4,096, runs of R <= 1/2 and R > 1/2, lengths capped at 32"}
    Nc, pc = N // 4, per * 4
    S, B, H = 1 << 14, 1 << 20, 256
    hist = torch.zeros(H, dtype=torch.int64, device="cuda")
    ms = timed(torch, stream, lambda: ph.phprng_collision_test(ctx, 0, Nc, pc, S, B, H, hist, stream), 4)
    torch.cuda.synchronize()
    got = hist.cpu().numpy()
    mean = float((got * np.arange(H)).sum() / max(got.sum(), 1))
    out["collision"] = {"value": Nc * pc / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
                        "workload": "plain32 first 16,384 instances x 16,384, segments of 2^14 into 2^20 bins",
                        "mean_collisions": mean,
                        "expected_mean": S - B * (1.0 - (1.0 - 1.0 / B) ** S)}
    return out


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


FP64_FMA_PER_CLK_SM = 2      # GB300's FP64 unit: 2 fused multiply-adds per clock per SM


def mode_fourier(ph, torch, stream, lgM=20):
    """The Fourier test at the paper's M = 2^20: 256 streams x 2^20 numbers
    (2^28 numbers, 256 sequences), real and imaginary parts into 8,192 bins
    over [-2, 2).  The FFT is bound by the FP64 unit; its achieved rate counts
    the conventional 2.5 M log2 M flops of a real transform of M points over
    the call's time minus that of generating the same numbers (timed alone)."""
    from paper_1411_2484_gb300 import workloads
    N, per, M = 256, 1 << 20, 1 << lgM
    inst = workloads.workload_instances("plain32_65536x4096x64", N)
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
    try:
        hist = torch.zeros(8192, dtype=torch.int64, device="cuda")
        ms = timed(torch, stream, lambda: ph.phprng_fourier_test(ctx, 0, N, per, lgM, 8192, 2.0, hist,
                                                                  None, stream), 4)
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        ms_gen = timed(torch, stream, lambda: ph.phprng_generate(ctx, 0, N, per, None, r, None, stream), 4)
    finally:
        ph.phprng_destroy(ctx)
    torch.cuda.synchronize()
    h = hist.cpu().numpy().astype(np.float64)
    centre = -2.0 + (np.arange(8192) + 0.5) * (4.0 / 8192)
    var = float((h * centre ** 2).sum() / h.sum() - ((h * centre).sum() / h.sum()) ** 2)
    flops = 2.5 * M * lgM * (N * per // M)
    peak = SMS * FP64_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fft_ms = max(ms - ms_gen, 1e-6)
    achieved = flops / fft_ms / 1e9
    return {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms, "ms_generate_alone": ms_gen,
            "workload": "256 streams x 2^20 numbers, M = 2^20 (the paper's), 8,192 bins over [-2, 2)",
            "variance_x24": var * 24,
            "roofline": {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz (unit counts x max clock)",
                         "algorithmic_flops_per_call": flops}}


def mode_wide64(ph, torch, stream, peak):
    from paper_1411_2484_gb300 import workloads
    inst = workloads.workload_instances("wide64_4096x2^20")
    N, per = 4096, 1 << 16
    ctx = ph.phprng_create(64, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
    try:
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        ms = timed(torch, stream, lambda: ph.phprng_generate(ctx, 0, N, per, None, r, None, stream),
                   4, warmup=1)
    finally:
        ph.phprng_destroy(ctx)
    muls = sum(muls_per_number(e, True) for e in inst["e"]) * per
    achieved = muls / (ms * 1e-3) / 1e12
    return {"value": N * per / ms * 1e3, "unit": "PRNs/s", "ms_per_call": ms,
            "workload": "4,096 64-bit safe primes x 2^16 numbers per call (R, 2 GiB)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T mul32/s",
                         "frac": achieved / peak}}


def mode_batched(ph, torch, stream, peak):
    """20,000 instances (16,000 32-bit, 4,000 64-bit), log-uniform lengths in
    [1, 2^20], offsets in [0, 2^40): one graph-replayed persistent launch
    (autotuned) against one skip+generate launch pair per request, all
    requests issued back to back on one stream."""
    from paper_1411_2484_gb300 import workloads
    w = workloads.WORKLOADS["batched_20000_mixed"]
    i32 = ph.phprng_draw_instances(32, w["instances32"], w["seed"], ph.PHPRNG_REQUIRE_SAFE_PRIME)
    i64 = ph.phprng_draw_instances(64, w["instances64"], w["seed"] + 1, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    inst = workloads.concat_instances(i32, i64)
    reqs = workloads.batched_requests(w["instances32"], w["instances64"], w["max_len"],
                                      w["max_offset"], w["seed"] + 2)
    total = int(reqs["len"].sum())
    # algorithmic multiply halves of the batch (the same count as the plain
    # launches: binary method + skip, 4 halves per 32-bit product, 20 per
    # 64-bit one); the skip-ahead to each offset is overhead, not counted
    e_all = np.concatenate([np.asarray(i32["e"], dtype=np.uint64), np.asarray(i64["e"], dtype=np.uint64)])
    wide = np.concatenate([np.zeros(len(i32["e"]), bool), np.ones(len(i64["e"]), bool)])
    muls = 0
    for (i, off, ln, _, _) in reqs:
        muls += muls_per_number(int(e_all[int(i)]), bool(wide[int(i)])) * int(ln)
    ctx = ph.phprng_create(0, inst, 0, stream)
    out = {}
    try:
        r = torch.empty(total, dtype=torch.float64, device="cuda")
        plan = ph.phprng_plan_create(ctx, reqs, 0, stream)
        try:
            tune = ph.phprng_plan_autotune(plan, None, r, stream, ctx=ctx)
            ms = timed(torch, stream, lambda: ph.phprng_plan_launch_graph(plan, None, r, stream,
                                                                          ctx=ctx), 5)
        finally:
            ph.phprng_plan_destroy(plan)
        achieved = muls / (ms * 1e-3) / 1e12
        out = {"value": total / ms * 1e3, "unit": "PRNs/s", "ms_per_launch": ms,
               "numbers": total, "requests": len(reqs), "tuning": tune,
               "numbers_32bit": int(reqs["len"][~wide[reqs["inst"].astype(np.int64)]].sum()),
               "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T mul32/s",
                            "frac": achieved / peak, "algorithmic_muls_per_launch": muls,
                            "peak_source": "152 SMs x 64 IMAD/clk x 2070 MHz (unit counts x max clock)"},
               "latency_ms": {"p50": ms, "p99": ms,
                              "note": "all requests are submitted together; each completes "
                                      "within the one launch, so completion since submission "
                                      "is at most the launch time"}}
    finally:
        ph.phprng_destroy(ctx)
    # one skip + generate launch pair per request, all 20,000 issued back to
    # back on one stream (no host synchronisation in between); CUDA events
    # around every pair give each request's own GPU time and its completion
    # time since the first submission
    ctx = ph.phprng_create(0, inst, 0, stream)
    try:
        r = torch.empty(int(reqs["len"].max()), dtype=torch.float64, device="cuda")
        ph.phprng_skip(ctx, [0], [1], stream)                 # builds the prefix table
        torch.cuda.synchronize()
        k = len(reqs)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for q, (i, off, ln, _, _) in enumerate(reqs):
            ev[q][0].record(stream)
            ph.phprng_skip(ctx, [int(i)], [int(off)], stream)
            ph.phprng_generate(ctx, int(i), 1, int(ln), None, r, None, stream)
            ev[q][1].record(stream)
        issue_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(ev[-1][1])
        own = np.array([a.elapsed_time(b) for a, b in ev])
        done = np.array([e0.elapsed_time(b) for _, b in ev])
        out["per_instance_launches"] = {
            "value": total / total_ms * 1e3, "unit": "PRNs/s", "requests": k,
            "ms_total": total_ms, "host_issue_s": issue_s,
            "service_ms": {"p50": float(np.percentile(own, 50)), "p99": float(np.percentile(own, 99))},
            "completion_since_submit_ms": {"p50": float(np.percentile(done, 50)),
                                           "p99": float(np.percentile(done, 99))},
            "note": "all 20,000 requests, skip + generate per request, issued back to back; "
                    "service = the request's own two launches, completion = since the first "
                    "submission"}
        out["batched_over_per_instance"] = out["value"] / out["per_instance_launches"]["value"]
    finally:
        ph.phprng_destroy(ctx)
    return out


def mode_served(ph, torch, duration_s=10.0, warm_s=1.0, rate=50000.0, tile=0, capacity=None):
    """1,000,000 32-bit streams, open-loop Poisson arrivals at 50k requests/s,
    sizes min(round(lognormal(ln 4096, 2)), 2^22), admission bounded by 16 GiB
    of outputs; PRNs/s and p50/p99 latency from arrival to completion."""
    rng = np.random.default_rng(4096)
    ctx = ph.phprng_create_seeded(32, 1_000_000, 0x5EED0004, ph.PHPRNG_REQUIRE_SAFE_PRIME)
    srv = None
    try:
        srv = ph.phprng_server_create(ctx, 16 << 30, max_batch=4096, inflight=4, tile=tile)
        span = warm_s + duration_s
        n = int(rate * span * 1.05) + 100
        gaps = rng.exponential(1.0 / rate, n)
        t = np.cumsum(gaps)
        t = t[t < span]
        n = t.size
        sizes = np.minimum(np.maximum(np.round(rng.lognormal(np.log(4096), 2.0, n)), 1),
                           1 << 22).astype(np.int64)
        streams = rng.integers(0, 1_000_000, n)
        t0 = ph.phprng_clock_ns() + 200_000_000
        arrivals = t0 + (t * 1e9).astype(np.int64)
        ph.phprng_server_submit(srv, streams, sizes, np.arange(n), arrivals)
        lat = np.zeros(n, dtype=np.int64)
        arr = np.zeros(n, dtype=np.int64)
        got = 0
        deadline = time.time() + span + 60
        while got < n and time.time() < deadline:
            comp = ph.phprng_server_poll(srv, 65536, 50_000_000)
            if len(comp):
                tags = comp["tag"].astype(np.int64)
                lat[tags] = comp["done_ns"] - comp["arrival_ns"]
                arr[tags] = comp["arrival_ns"]
                got += len(comp)
                ph.phprng_server_release(srv, comp["id"])
        st = ph.phprng_server_stats_get(srv)
    finally:
        if srv:
            ph.phprng_server_destroy(srv)
        ph.phprng_destroy(ctx)
    meas = (arrivals >= t0 + int(warm_s * 1e9))
    l_ms = lat[meas] / 1e6
    numbers = int(sizes[meas].sum())
    offered = float(sizes[meas].sum()) / duration_s
    return {"value": numbers / duration_s, "unit": "PRNs/s",
            "roofline": {"bound": "offered_load", "achieved": numbers / duration_s, "peak": offered,
                         "unit": "PRNs/s", "frac": numbers / duration_s / offered,
                         "capacity_prn_s": capacity,
                         "offered_over_capacity": offered / capacity if capacity else None,
                         "note": "open-loop arrivals: the server completes what arrives, so its "
                                 "throughput is the offered load; capacity = the plain launch's "
                                 "measured rate on the same GPU"},
            "requests": int(meas.sum()), "completed": int(got),
            "latency_ms": {"p50": float(np.percentile(l_ms, 50)),
                           "p99": float(np.percentile(l_ms, 99)),
                           "max": float(l_ms.max())},
            "offered_rate_req_s": rate, "batches": st["batches"], "tile": tile,
            "max_waiting": st["max_waiting"],
            "workload": "1,000,000 32-bit streams, Poisson 50k req/s, lognormal(ln 4096, 2) "
                        "sizes capped at 2^22, 16 GiB admission, R only"}


def run_reference(args, rank):
    """Times the CPU oracle (the reference arm) on rank 0."""
    if rank != 0:
        return
    import oracle
    from paper_1411_2484_gb300 import workloads
    w = workloads.WORKLOADS[WORKLOAD]
    per = w["per_inst"]
    inst = workloads.workload_instances(WORKLOAD, count=1024)
    rows = workloads.instance_rows(inst)
    cores = host_cores()
    for _ in range(args.warmup):
        oracle.generate_many(rows[:cores], per, threads=cores, want_c=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.generate_many(rows, per, threads=cores, want_c=False)
    dt = time.perf_counter() - t0
    value = args.steps * len(rows) * per / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "PRNs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": len(rows), "per_inst": per,
                   "step": "1,024 of the 65,536 instances x 4,096 numbers (R stored) per step"},
        "cpu_baseline": {"value": value, "unit": "PRNs/s", "cores": cores, "kind": "oracle",
                         "sample": "1,024 instances x 4,096 numbers per step, %d steps"
                                   % args.steps},
        "e2e": {"value": value, "unit": "PRNs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def rank_instances(workloads, w, rank, world):
    """The instances of one rank: its own seeded draw of w["instances"] safe
    primes from its own slice of [2^31, 2^32), so that moduli stay distinct
    across ranks (parameter splitting) with no exchange between ranks.  One
    rank draws exactly the single-GPU workload."""
    lo, hi = 1 << 31, 1 << 32
    span = (hi - lo) // world
    top = hi if rank == world - 1 else lo + (rank + 1) * span
    return workloads.draw_instances(w["instances"], width=32, seed=w["seed"] + 7919 * rank,
                                    n_range=(lo + rank * span, top), exponent=w.get("exponent"))


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values of x (all ranks get it)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_1411_2484_gb300 as ph
    from paper_1411_2484_gb300 import workloads

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    w = workloads.WORKLOADS[WORKLOAD]
    N, per = w["instances"], w["per_inst"]
    inst = rank_instances(workloads, w, rank, world)
    stream = torch.cuda.current_stream()
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
    r = torch.empty(N * per, dtype=torch.float64, device="cuda")

    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler("GPU-" + str(uuid) if uuid else None)
    time.sleep(0.3)                                   # the sampler's own start-up
    for _ in range(args.warmup):
        ph.phprng_generate(ctx, 0, N, per, None, r, None, stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    start.record(stream)
    for _ in range(args.steps):
        ph.phprng_generate(ctx, 0, N, per, None, r, None, stream)
    end.record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop(wall0, wall1)
    ms = max_over_ranks(start.elapsed_time(end), dist, "cuda")
    numbers = args.steps * N * per * world
    value = numbers / (ms / 1e3)

    # e2e: the same call with a pinned host output buffer (copies inside)
    steps_e2e = min(args.steps, 8)
    r_host = torch.empty(N * per, dtype=torch.float64, pin_memory=True)
    ph.phprng_generate(ctx, 0, N, per, None, r_host, None, stream)      # warm staging
    # three timed runs of steps_e2e calls; the median run is reported (the
    # host clock sees the occasional slow run of the host's own work)
    runs = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            ph.phprng_generate(ctx, 0, N, per, None, r_host, None, stream)
        runs.append(max_over_ranks(time.perf_counter() - t0, dist, "cuda"))
    dt = sorted(runs)[1]
    # the link's own rate on this host: plain copies of the same bytes into the same buffer
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(4):
        r_host.copy_(r, non_blocking=True)
    torch.cuda.synchronize()
    link = 4 * N * per * 8 / (time.perf_counter() - t0) / 1e9
    e2e = {"value": steps_e2e * N * per * world / dt, "unit": "PRNs/s",
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": N * per * 8,
           "steps": steps_e2e, "runs": 3, "run_s": runs, "reported": "median run", "d2h_link_gbs": link,
           "link_bound_prn_s": link * 1e9 / 8 * world}

    ph.phprng_destroy(ctx)
    if rank != 0:
        return
    muls = algorithmic_muls(inst["e"], per)
    launch_s = ms / 1e3 / args.steps
    achieved = muls / launch_s / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "PRNs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": N, "per_inst": per,
                   "output": "R_k FP64 to HBM, 2 GiB per step", "seed": w["seed"],
                   "l2": "no flush: each step writes 2 GiB of outputs (> 129 MB L2)",
                   "parallelism": "independent instances per GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": PEAK_TMULS,
                     "unit": "T mul32/s", "frac": achieved / PEAK_TMULS,
                     "traffic": profile_traffic("gen32_kernel"),
                     "kernel": "gen32_kernel",
                     "ncu_inst_per_number": (profile_entry("gen32_kernel") or {}).get("ncu_inst_per_number"),
                     "algorithmic_muls_per_number": muls / (N * per),
                     "peak_source": "152 SMs x 64 IMAD/clk x 2070 MHz (unit counts x max clock)",
                     "algorithmic_muls_per_launch": muls},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if world == 1:
        out["cpu_baseline"] = cpu_baseline(inst, per)
        modes = {}
        wanted = [] if args.modes == "none" else args.modes.split(",")
        for name, fn in (("fused", lambda: mode_fused(ph, torch, ctx2, N, per, stream, 8)),
                         ("serial", lambda: mode_serial(ph, torch, ctx2, N, per, stream)),
                         ("interstream", lambda: mode_interstream(ph, torch, ctx2, N, per, stream)),
                         ("consumers", lambda: mode_consumers(ph, torch, ctx2, N, per, stream)),
                         ("small_e", lambda: mode_small_e(ph, torch, stream, PEAK_TMULS)),
                         ("pattern", lambda: mode_pattern(ph, torch, stream)),
                         ("fourier", lambda: mode_fourier(ph, torch, stream)),
                         ("figures", lambda: mode_figures(ph, torch, stream)),
                         ("wide64", lambda: mode_wide64(ph, torch, stream, PEAK_TMULS)),
                         ("c0", lambda: mode_c0(ph, torch, stream, PEAK_TMULS)),
                         ("batched", lambda: mode_batched(ph, torch, stream, PEAK_TMULS)),
                         ("served", lambda: mode_served(ph, torch, capacity=value))):
            if name not in wanted:
                continue
            try:
                if name in ("fused", "serial", "interstream", "consumers"):
                    ctx2 = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
                    try:
                        modes[name] = fn()
                    finally:
                        ph.phprng_destroy(ctx2)
                else:
                    modes[name] = fn()
            except Exception as exc:                   # a mode never hides the headline
                modes[name] = {"error": repr(exc)[:300]}
        out["modes"] = modes
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
