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
    """nvidia-smi samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.proc = None
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if uuid:
                cmd += ["-i", uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def profile_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
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
    return d.get("bytes_per_launch")


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
    return {"value": count * per_inst / dt, "unit": "PRNs/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of the %d instances x %d numbers (R stored), %.1f s"
                      % (count, len(rows), per_inst, dt)}


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
    inst = workloads.draw_instances(N, width=32, seed=w["seed"] + 7919 * rank)
    stream = torch.cuda.current_stream()
    ctx = ph.phprng_create(32, inst, ph.PHPRNG_REQUIRE_SAFE_PRIME, stream)
    r = torch.empty(N * per, dtype=torch.float64, device="cuda")

    for _ in range(args.warmup):
        ph.phprng_generate(ctx, 0, N, per, None, r, None, stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler("GPU-" + str(uuid) if uuid else None)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        ph.phprng_generate(ctx, 0, N, per, None, r, None, stream)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = start.elapsed_time(end)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    numbers = args.steps * N * per * world
    value = numbers / (ms / 1e3)

    # e2e: the same call with a pinned host output buffer (copies inside)
    steps_e2e = min(args.steps, 8)
    r_host = torch.empty(N * per, dtype=torch.float64, pin_memory=True)
    ph.phprng_generate(ctx, 0, N, per, None, r_host, None, stream)      # warm staging
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps_e2e):
        ph.phprng_generate(ctx, 0, N, per, None, r_host, None, stream)
    dt = time.perf_counter() - t0
    if dist:
        t = torch.tensor([dt], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    e2e = {"value": steps_e2e * N * per * world / dt, "unit": "PRNs/s",
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": N * per * 8,
           "steps": steps_e2e}

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
                     "peak_source": "152 SMs x 64 IMAD/clk x 2070 MHz (unit counts x max clock)",
                     "algorithmic_muls_per_launch": muls},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if world == 1:
        out["cpu_baseline"] = cpu_baseline(inst, per)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
