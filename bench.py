#!/usr/bin/env python3
"""Benchmark of GPU system calls on B300 (one JSON line on stdout).

Workload (one step): the invocation microbenchmark sweep - 2^10 .. 2^20 GPU
threads, each writing its 64-byte splitmix64 pattern to a tmpfs file with
pwrite at offset gid*64, at every legal combination of granularity
{work-item, warp, work-group of 64/256/1024, kernel} x ordering {strong,
relaxed} x blocking {blocking, non-blocking} (22 combinations, 132 kernels)
- followed by the C1 pread pass (a 4 MiB file read in 4 KiB preads by 64
work-groups of 256 threads into a 256-bin histogram, plain and batched).

value = GPU system calls retired per second over the step (device-event
timing around the whole step; every entry point synchronises and drains, so
the step's calls are all complete inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl genesys|reference]

--impl reference times the CPU oracle (a sequential C program issuing the
same pwrite/pread calls) on the same workload on the host cores.
Multi-GPU: independent replicas (the sweep has no exchange step), one rank per
GPU, max time over ranks, value = all ranks' calls / that time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIZES = [1 << 10, 1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 20]
GRAINS = [  # name, GENESYS_GRAN_*, threads per block
    ("work-item", 0, 256), ("warp", 1, 256), ("wg64", 2, 64), ("wg256", 2, 256), ("wg1024", 2, 1024),
    ("kernel", 3, 256)]
COMBOS = [(name, g, bt, relaxed, nb) for name, g, bt in GRAINS for relaxed in (False, True) for nb in (False, True)
          if not (g == 0 and relaxed)]
SEED_C2 = 0x5EED0002
C1_BYTES, C1_CHUNK, C1_GROUPS, C1_THREADS = 4 << 20, 4096, 64, 256
SCAN_BYTES, SCAN_CHUNK, SCAN_GROUPS, SCAN_THREADS = 1 << 30, 1 << 20, 148, 1024
SERVICE_THREADS = 4


def combo_key(name, relaxed, nb):
    return f"{name}/{'relaxed' if relaxed else 'strong'}/{'nonblocking' if nb else 'blocking'}"


def calls_for(gran, bt, n):
    if gran == 0:
        return n
    if gran == 1:
        return -(-n // 32)
    if gran == 2:
        return -(-n // bt)
    return 1


def step_calls():
    c2 = sum(calls_for(g, bt, n) for n in SIZES for _, g, bt, _, _ in COMBOS)
    c1 = 2 * (C1_BYTES // C1_CHUNK)
    return c2, c1


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{gpu}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path).read().splitlines()[1:]:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1].split()[0]))
                mx = float(parts[2].split()[0])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


# ---------------------------------------------------------------- helpers
def host_link_peak(torch):
    """Pinned cudaMemcpy H2D / D2H bandwidth at 256 MiB (best of 5), GB/s."""
    n = 256 << 20
    h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = {}
    for name, (dst, src) in {"h2d": (d, h), "d2h": (h, d)}.items():
        best = 0.0
        for _ in range(6):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            dst.copy_(src, non_blocking=True)
            e.record()
            e.synchronize()
            best = max(best, n / (s.elapsed_time(e) * 1e-3) / 1e9)
        out[name] = round(best, 2)
    del h, d
    return out


def pctl(a, q):
    import numpy as np
    return float(np.percentile(a, q)) if len(a) else None


def load_traffic(kernel: str):
    """ncu host-link traffic (bytes per launch) for `kernel` from the committed
    profile summary, or None if the kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha1()
    for f in ("paper_1705_06965_b300/csrc/workloads.cu", "include/genesys_device.cuh"):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    src = h.hexdigest()[:12]
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == src:
            return float(parts[2])
    return None


# ---------------------------------------------------------------- GPU arm
def run_genesys(args):
    import numpy as np
    import torch

    import paper_1705_06965_b300 as G
    import workloads

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    d = workloads.scratch_dir(f"bench_r{rank}")
    c1_path = workloads.c1_file(os.path.join(d, "c1.bin"), C1_BYTES, seed=workloads.SEED_C1)
    scan_path = workloads.c1_file(os.path.join(d, "scan.bin"), SCAN_BYTES, seed=0x5EED00F1)
    ctx = G.Context(device=local, service_threads=SERVICE_THREADS, staging_bytes=400 << 20,
                    deadline_ns=10_000_000_000)
    c2_stage = ctx.staging(max(SIZES) * 64)
    c1_stage = ctx.staging(max(2 * C1_GROUPS * C1_CHUNK, 2 * SCAN_GROUPS * SCAN_CHUNK))
    c1_stage_bytes = max(2 * C1_GROUPS * C1_CHUNK, 2 * SCAN_GROUPS * SCAN_CHUNK)
    fds = {n: os.open(os.path.join(d, f"c2_{n}.bin"), os.O_CREAT | os.O_RDWR, 0o644) for n in SIZES}
    fd_c1 = os.open(c1_path, os.O_RDONLY)
    fd_scan = os.open(scan_path, os.O_RDONLY)
    hist = torch.zeros((2, 256), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    kernel_ms = {}
    launches = [0]

    def note(kname):
        kernel_ms.setdefault(kname, []).append(ctx.last_launch_ms())
        launches[0] += 1

    def one_step(collect_kernels=True):
        for n in SIZES:
            for name, g, bt, relaxed, nb in COMBOS:
                ctx.c2_pwrite(fds[n], n, g, bt, relaxed, nb, SEED_C2, c2_stage, n * 64)
                if collect_kernels:
                    note(f"c2_pwrite_kernel<{G.GRAN_NAMES[g]},{'relaxed' if relaxed else 'strong'},"
                         f"{'nonblocking' if nb else 'blocking'}>")
        for form in (G.FORM_PLAIN, G.FORM_BATCHED):
            ctx.c1_histogram(fd_c1, C1_BYTES, hist[form].data_ptr(), c1_stage, c1_stage_bytes, chunk=C1_CHUNK,
                             groups=C1_GROUPS, threads=C1_THREADS, form=form)
            if collect_kernels:
                note("c1_plain_kernel" if form == G.FORM_PLAIN else "c1_batched_kernel")

    # warm-up (untimed)
    for _ in range(max(args.warmup, 0)):
        hist.zero_()
        one_step(collect_kernels=False)
    torch.cuda.synchronize()
    kernel_ms.clear()
    launches[0] = 0
    ctx.stats_reset()

    c2_calls, c1_calls = step_calls()
    step_ms, e2e_s = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps
            hist.zero_()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            one_step()
            e.record(stream)
            h = hist.cpu()                     # the step's result back on the host
            st = ctx.status()
            e.synchronize()
            e2e_s.append(time.perf_counter() - t0)
            step_ms.append(s.elapsed_time(e))
            if any(st):
                raise RuntimeError(f"device status {st}")
    stats = ctx.stats()
    clocks = clk.summary()

    # correctness spot check outside the timed region (parity tests cover it in full)
    import oracle
    want = oracle.c1_histogram(c1_path, C1_CHUNK)
    if not (np.array_equal(h[0].numpy().view(np.uint32), want) and np.array_equal(h[1].numpy().view(np.uint32), want)):
        raise RuntimeError("C1 histogram differs from the oracle")

    tot_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_ms, sum(e2e_s)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms, e2e_tot = float(t[0]), float(t[1])
    else:
        e2e_tot = sum(e2e_s)
    calls_step = c2_calls + c1_calls
    value = world * calls_step * args.steps / (tot_ms * 1e-3)

    # ---- profile pass (untimed): per-combination rate and latency at 2^20,
    # plain vs batched forms, pread+scan GB/s at 1 GiB
    sweep = {}
    n = max(SIZES)
    for name, g, bt, relaxed, nb in COMBOS:
        ctx.latency(clear=True)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        ctx.c2_pwrite(fds[n], n, g, bt, relaxed, nb, SEED_C2, c2_stage, n * 64)
        e.record(stream)
        e.synchronize()
        ms = s.elapsed_time(e)
        lat = ctx.latency(clear=True)
        calls = calls_for(g, bt, n)
        sweep[combo_key(name, relaxed, nb)] = {
            "ms": round(ms, 3), "syscalls_per_s": round(calls / (ms * 1e-3), 1),
            "requests_per_s": round(n / (ms * 1e-3), 1),
            "p50_us": round(pctl(lat, 50) / 1e3, 2) if len(lat) else None,
            "p99_us": round(pctl(lat, 99) / 1e3, 2) if len(lat) else None}
    plain = sweep[combo_key("work-item", False, False)]
    batched = max((v for k, v in sweep.items() if "relaxed" in k), key=lambda v: v["requests_per_s"])
    batched_key = [k for k, v in sweep.items() if v is batched][0]

    link = host_link_peak(torch)
    scan = {}
    for form in (G.FORM_PLAIN, G.FORM_BATCHED):
        ctx.stats_reset()
        best = None
        for _ in range(3):
            hist.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            ctx.c1_histogram(fd_scan, SCAN_BYTES, hist[0].data_ptr(), c1_stage, c1_stage_bytes, chunk=SCAN_CHUNK,
                             groups=SCAN_GROUPS, threads=SCAN_THREADS, form=form)
            e.record(stream)
            e.synchronize()
            ms = s.elapsed_time(e)
            best = ms if best is None else min(best, ms)
        gbs = SCAN_BYTES / (best * 1e-3) / 1e9
        scan["plain" if form == G.FORM_PLAIN else "batched"] = {
            "GB_per_s": round(gbs, 2), "frac_of_host_link_h2d": round(gbs / link["h2d"], 4), "ms": round(best, 2)}

    # dominant kernel of the timed region and its host-link roofline
    tot = {k: sum(v) for k, v in kernel_ms.items()}
    dom = max(tot, key=tot.get)
    avg_ms = statistics.mean(kernel_ms[dom])
    # algorithmic host-link bytes per launch of the dominant kernel, averaged
    # over the sizes it ran at: per GPU thread its 64-byte payload written to
    # pinned memory; per call a 64-byte slot + 8-byte doorbell written and an
    # 8-byte completion word read.
    if dom.startswith("c2_pwrite_kernel"):
        gname = dom.split("<")[1].split(",")[0]
        gr = {v: k for k, v in G.GRAN_NAMES.items()}[gname]
        per = []
        for nn in SIZES:
            for name, g, bt, relaxed, nb in COMBOS:
                if g == gr and f"{'relaxed' if relaxed else 'strong'}" in dom and (
                        ("nonblocking" in dom) == nb):
                    per.append(nn * 64 + calls_for(g, bt, nn) * 80)
        alg_bytes = statistics.mean(per)
    else:
        alg_bytes = C1_BYTES + (C1_BYTES // C1_CHUNK) * 80
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    peak = link["d2h"] if dom.startswith("c2") else link["h2d"]
    roofline = {"bound": "host_link", "kernel": dom, "achieved": round(achieved, 3), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 5), "traffic": load_traffic(dom),
                "peak_source": "pinned cudaMemcpy 256 MiB in this run (of measured)",
                "alg_bytes_per_launch": int(alg_bytes), "avg_launch_ms": round(avg_ms, 4),
                "share_of_timed_device_time": round(tot[dom] / sum(tot.values()), 4)}

    # CPU baseline: the oracle as it stands, on this host, bounded sample
    cpu = None
    if rank == 0:
        cpu = cpu_baseline_sample(budget_s=20.0)

    lat_all = []
    line = {
        "metric": "GPU syscalls/s (C2 pwrite invocation sweep + C1 pread pass)",
        "value": round(value, 1), "unit": "syscalls/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "C2 invocation microbenchmark sweep: 2^10..2^20 threads x {work-item, warp, "
                               "work-group 64/256/1024, kernel} x {strong, relaxed} x {blocking, non-blocking}, "
                               "64-byte pwrite per thread to a tmpfs file at gid*64; then C1 (4 MiB file, 4 KiB "
                               "preads, 64 work-groups x 256 threads, 256-bin histogram, plain and batched)",
                   "threads": SIZES, "combinations": len(COMBOS), "kernels_per_step": len(SIZES) * len(COMBOS) + 2,
                   "syscalls_per_step": calls_step, "service_threads": SERVICE_THREADS,
                   "l2": "256 MiB device buffer written between timed steps (L2 flush)",
                   "parallelism": f"replicas x{world}"},
        "requests_per_s": round(world * (sum(SIZES) * len(COMBOS) + c1_calls) * args.steps / (tot_ms * 1e-3), 1),
        "forms": {"plain_blocking_strong": {"combo": "work-item/strong/blocking", **plain},
                  "batched": {"combo": batched_key, **batched}},
        "sweep_2p20": sweep,
        "pread_scan_1GiB": scan,
        "host_link_GB_per_s": link,
        "service": {k: stats[k] for k in ("requests", "os_calls", "batches", "bytes", "failed")},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(world * calls_step * args.steps / e2e_tot, 1), "unit": "syscalls/s",
                "h2d_bytes_per_step": 2 * C1_BYTES,
                "d2h_bytes_per_step": sum(SIZES) * 64 * len(COMBOS) + 2 * 1024 + 32},
        "clocks": clocks,
        "gpu_launches": launches[0],
    }
    del lat_all
    for fd in list(fds.values()) + [fd_c1, fd_scan]:
        os.close(fd)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- oracle
def oracle_step(d, budget_s=None):
    """One step of the workload by the CPU oracle: the same sweep of pwrites
    (grouped as each granularity issues them) and the C1 preads.  Returns
    (syscalls, seconds)."""
    import oracle
    import workloads
    c1_path = workloads.c1_file(os.path.join(d, "c1.bin"), C1_BYTES, seed=workloads.SEED_C1)
    calls, t0 = 0, time.perf_counter()
    for n in SIZES:
        p = os.path.join(d, f"c2o_{n}.bin")
        for name, g, bt, relaxed, nb in COMBOS:
            group = {0: 1, 1: 32, 2: bt, 3: n}[g]
            calls += oracle.c2_pwrite(p, n, group, SEED_C2)
            if budget_s and time.perf_counter() - t0 > budget_s:
                return calls, time.perf_counter() - t0, False
    for _ in range(2):
        oracle.c1_histogram(c1_path, C1_CHUNK)
        calls += C1_BYTES // C1_CHUNK
    return calls, time.perf_counter() - t0, True


def cpu_baseline_sample(budget_s=20.0):
    import workloads
    d = workloads.scratch_dir("bench_oracle")
    calls, sec, full = oracle_step(d, budget_s)
    return {"value": round(calls / sec, 1), "unit": "syscalls/s", "cores": 1, "kind": "oracle",
            "sample": ("one full step" if full else f"first {calls} calls of one step") +
                      " (C2 sweep + C1 preads), sequential C oracle, 1 thread",
            "host_cpus": os.cpu_count()}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import workloads
    d = workloads.scratch_dir("bench_reference")
    for _ in range(max(args.warmup, 0)):
        oracle_step(d)
    tot_calls, tot_s = 0, 0.0
    for _ in range(args.steps):
        c, s, _ = oracle_step(d)
        tot_calls += c
        tot_s += s
    v = tot_calls / tot_s
    line = {"impl": "reference", "metric": "GPU syscalls/s (C2 pwrite invocation sweep + C1 pread pass)",
            "value": round(v, 1), "unit": "syscalls/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_s * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "same sweep and pread pass, issued by the sequential CPU oracle",
                       "syscalls_per_step": sum(step_calls())},
            "cpu_baseline": {"value": round(v, 1), "unit": "syscalls/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full steps"},
            "e2e": {"value": round(v, 1), "unit": "syscalls/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="genesys", choices=["genesys", "reference"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_genesys(args)


if __name__ == "__main__":
    main()
