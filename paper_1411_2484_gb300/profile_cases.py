"""Single launches of each kernel on fixed, moderately sized cases, for ncu.

    python -m paper_1411_2484_gb300.profile_cases CASE [--repeat N]

CASE is one of
  plain32   65,536 instances x 4,096 numbers, R to HBM (2 GiB)     gen32_kernel
  c0        4 safe 32-bit instances x 2^20 numbers, c and R stored
            (a split launch: chunk_sums_kernel, then gen32_kernel)
  fused32   the same instances, statistics only                      gen32_kernel (STATS)
  small_e   65,536 instances with e = 9 x 4,096 numbers, R (2 GiB)   gen32_kernel
  serial2   plain32's instances, pairs into 2^20 bins (serial test)  serial_kernel
  pattern3  the paper's pattern instance (n = 4294967087, p = 2^31-1,
            e = 9), D = 3, 2^24 volumes, L0 = 4 (2^33 points)       pattern_kernel
  wide64    4,096 64-bit instances x 4,096 numbers, R (128 MiB)      gen64_kernel
  collision plain32's first 16,384 instances x 16,384 numbers, segments
            of 2^14 into 2^20 bins (the paper's collision test)      coll_bins_kernel,
                                                                      coll_count_kernel
  inter2    plain32's instances, interleaved order (number 1 of every
            stream, then number 2 ...), pairs into 2^20 bins          inter_*_kernel
  fourier20 plain32's first 256 instances x 2^20 numbers, Fourier test
            over sequences of M = 2^20 (the paper's), 8,192 bins       fft_*_kernel
  batched   2,000 instances (80 % 32-bit), lengths log-uniform in
            [1, 2^18], offsets in [0, 2^40), R (about 0.4 GiB)       batch_kernel
  batched20k  the batched bench workload's 20,000 instances (16,000
            32-bit, 4,000 64-bit) and offsets, lengths log-uniform in
            [1, 2^20] (--max-len, default the bench's 2^20: 12 GiB of R;
            2^15 gives 0.5 GiB for multi-pass captures)              batch_kernel
Each case warms up once, then launches its kernel N times (default 3) and
prints the CUDA-event time per launch.  Inputs are the seeded workloads of
paper_1411_2484_gb300.workloads.
"""
import argparse
import json

import torch

import paper_1411_2484_gb300 as ph
from paper_1411_2484_gb300 import workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["plain32", "c0", "collision", "fused32", "small_e", "serial2", "pattern3", "wide64", "batched",
                                     "batched20k", "fourier20", "inter2"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--max-len", type=int, default=1 << 20)
    args = ap.parse_args()
    s = torch.cuda.current_stream()
    ctx, plan = None, None
    if args.case == "pattern3":
        hist = torch.zeros(1 << 24, dtype=torch.int64, device="cuda")
        run = lambda: ph.phprng_pattern(4294967087, 9, 2147483647, 784588716, 1000, 4, 3, 4096, hist, s)
        numbers = 4 * (2147483647 - 1) * 2                  # exponentiations
    elif args.case == "serial2":
        inst = workloads.workload_instances("plain32_65536x4096x64")
        N, per = 65536, 4096
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        hist = torch.zeros(1 << 20, dtype=torch.int64, device="cuda")
        run = lambda: ph.phprng_serial_test(ctx, 0, N, per, 2, 1 << 10, hist, s)
        numbers = N * per
    elif args.case in ("plain32", "fused32"):
        inst = workloads.workload_instances("plain32_65536x4096x64")
        N, per = 65536, 4096
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        if args.case == "plain32":
            r = torch.empty(N * per, dtype=torch.float64, device="cuda")
            run = lambda: ph.phprng_generate(ctx, 0, N, per, None, r, None, s)
        else:
            sb = torch.empty(N * ph.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            run = lambda: ph.phprng_generate(ctx, 0, N, per, None, None, sb, s)
        numbers = N * per
    elif args.case == "collision":
        inst = workloads.workload_instances("plain32_65536x4096x64", 16384)
        N, per = 16384, 16384
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        hist = torch.zeros(256, dtype=torch.int64, device="cuda")
        run = lambda: ph.phprng_collision_test(ctx, 0, N, per, 1 << 14, 1 << 20, 256, hist, s)
        numbers = N * per
    elif args.case == "c0":
        name = "pr1_ref_32bit_4x2^20"
        inst = workloads.workload_instances(name)
        N, per = workloads.WORKLOADS[name]["instances"], workloads.WORKLOADS[name]["per_inst"]
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        c = torch.empty(N * per, dtype=torch.int32, device="cuda")
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        run = lambda: ph.phprng_generate(ctx, 0, N, per, c, r, None, s)
        numbers = N * per
    elif args.case == "inter2":
        inst = workloads.workload_instances("plain32_65536x4096x64")
        N, per = 65536, 4096
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        hist = torch.zeros(1 << 20, dtype=torch.int64, device="cuda")
        run = lambda: ph.phprng_interstream_serial_test(ctx, 0, N, per, 2, 1 << 10, hist, s)
        numbers = N * per
    elif args.case == "fourier20":
        inst = workloads.workload_instances("plain32_65536x4096x64", 256)
        N, per = 256, 1 << 20
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        hist = torch.zeros(8192, dtype=torch.int64, device="cuda")
        run = lambda: ph.phprng_fourier_test(ctx, 0, N, per, 20, 8192, 2.0, hist, None, s)
        numbers = N * per
    elif args.case == "small_e":
        inst = workloads.workload_instances("plain32_e9_65536x4096")
        N, per = 65536, 4096
        ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        run = lambda: ph.phprng_generate(ctx, 0, N, per, None, r, None, s)
        numbers = N * per
    elif args.case == "wide64":
        inst = workloads.workload_instances("wide64_4096x2^20")
        N, per = 4096, 4096
        ctx = ph.phprng_create(64, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, s)
        r = torch.empty(N * per, dtype=torch.float64, device="cuda")
        run = lambda: ph.phprng_generate(ctx, 0, N, per, None, r, None, s)
        numbers = N * per
    elif args.case == "batched20k":
        w = workloads.WORKLOADS["batched_20000_mixed"]
        i32 = ph.phprng_draw_instances(32, w["instances32"], w["seed"], ph.PHPRNG_REQUIRE_SAFE_PRIME)
        i64 = ph.phprng_draw_instances(64, w["instances64"], w["seed"] + 1, ph.PHPRNG_REQUIRE_SAFE_PRIME)
        inst = workloads.concat_instances(i32, i64)
        reqs = workloads.batched_requests(w["instances32"], w["instances64"], args.max_len, w["max_offset"],
                                          w["seed"] + 2)
        numbers = int(reqs["len"].sum())
        ctx = ph.phprng_create(0, inst, 0, s)
        r = torch.empty(numbers, dtype=torch.float64, device="cuda")
        plan = ph.phprng_plan_create(ctx, reqs, 0, s)
        run = lambda: ph.phprng_plan_launch(plan, None, r, s, ctx=ctx)
    else:
        i32 = workloads.draw_instances(1600, seed=0x5EED0005)
        i64 = workloads.draw_instances(400, width=64, seed=0x5EED0006)
        inst = workloads.concat_instances(i32, i64)
        reqs = workloads.batched_requests(1600, 400, max_len=1 << 18, seed=0x5EED0007)
        numbers = int(reqs["len"].sum())
        ctx = ph.phprng_create(0, inst, 0, s)
        r = torch.empty(numbers, dtype=torch.float64, device="cuda")
        plan = ph.phprng_plan_create(ctx, reqs, 0, s)
        run = lambda: ph.phprng_plan_launch(plan, None, r, s, ctx=ctx)
    try:
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.repeat):
            run()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.repeat
        print(json.dumps({"case": args.case, "numbers": numbers, "ms_per_launch": ms,
                          "prn_s": numbers / ms * 1e3}))
    finally:
        if plan:
            ph.phprng_plan_destroy(plan)
        if ctx:
            ph.phprng_destroy(ctx)


if __name__ == "__main__":
    main()
