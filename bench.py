#!/usr/bin/env python3
"""Benchmark of GPU system calls on B300 (one JSON line on stdout).

Workload (one step): the invocation microbenchmark sweep - 2^10 .. 2^20 GPU
threads, each writing its 64-byte splitmix64 pattern to a tmpfs file with
pwrite at offset gid*64, at every legal combination of granularity
{work-item, warp, work-group of 64/256/1024, kernel} x ordering {strong,
relaxed} x blocking {blocking, non-blocking} (22 combinations, 132 kernels)
- followed by the C1 pread pass (a 4 MiB file read in 4 KiB preads by 64
work-groups of 256 threads into a 256-bin histogram, plain and batched).

value = GPU system calls retired per second over the step (CUDA-event timing
around the whole step; every entry point synchronises and drains, so the
step's calls are all complete inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl genesys|reference]
    python bench.py --only c2:work-item/strong/blocking:65536   # one case (profiling)
    python bench.py --only c1:batched:1073741824
    python bench.py --only c3:batched
    python bench.py --only c4          # key-value service rate sweep (+ oracle server)
    python bench.py --only c5          # the served mixed trace
    python bench.py --only c5:persistent:1000   # one serving form, first n requests
    python bench.py --only fig10       # echo bandwidth versus packet size
    python bench.py --only f4          # open/write/lseek/read/close/madvise from GPU code

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
ALG_BYTES_PER_CALL = 64 + 8  # a call's slot and its result word (payload bytes are counted apart)
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
C3_CHUNK, C3_CTAS, C3_THREADS = 1 << 20, 296, 512
GRAN_BY_NAME = {name: (g, bt) for name, g, bt in GRAINS}
PROFILE_REPEATS = 3  # runs of each combination in the untimed profile pass


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


# ---------------------------------------------------------------- replicas
def reduce_max(values, device=None):
    """Element-wise max of per-rank values over all ranks (identity with one
    rank).  Multi-GPU runs are independent replicas: the slowest rank's time
    is the job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_value(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / max_seconds


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None
        import tempfile
        # the raw samples: GENESYS_CLOCKS_DIR if set, else the temporary directory
        d = os.environ.get("GENESYS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"genesys_clocks_{os.getpid()}_{gpu}.csv")

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
def host_pwrite_peak(fd, buf, nbytes, repeats=3, chunks=(256 << 10, 1 << 20, 4 << 20, 64 << 20)):
    """Best GB/s of one host thread writing nbytes from host address buf to fd
    (offset 0 on) with pwrite calls of each chunk size, best of `repeats`;
    returns (GB/s, chunk)."""
    import ctypes
    libc = ctypes.CDLL(None, use_errno=True)
    libc.pwrite.restype = ctypes.c_ssize_t
    libc.pwrite.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_long]
    best, best_chunk = 0.0, None
    for chunk in chunks:
        for _ in range(repeats):
            t = time.perf_counter()
            done = 0
            while done < nbytes:
                r = libc.pwrite(fd, buf + done, min(chunk, nbytes - done), done)
                if r <= 0:
                    raise OSError(ctypes.get_errno(), "pwrite")
                done += r
            gbs = nbytes / (time.perf_counter() - t) / 1e9
            if gbs > best:
                best, best_chunk = gbs, chunk
    return best, best_chunk


def host_probes(torch, local, scan_path):
    """What the design depends on, measured on this machine: the host CPU, SM
    count, whether the GPU has native atomics on host memory (the protocol
    never needs them), and one host thread's tmpfs pread GB/s (1 MiB preads of
    the 1 GiB scan file into a reused buffer: the per-thread copy rate that
    sets how many service threads a scan needs)."""
    import platform
    import numpy as np
    out = {"machine": platform.machine(), "host_cpus": os.cpu_count(),
           "sm_count": torch.cuda.get_device_properties(local).multi_processor_count}
    try:
        with open("/proc/cpuinfo") as f:
            out["cpu_model"] = next((ln.split(":", 1)[1].strip() for ln in f if ln.startswith("model name")), None)
    except OSError:
        pass
    try:
        from cuda.bindings import runtime as rt
        err, v = rt.cudaDeviceGetAttribute(rt.cudaDeviceAttr.cudaDevAttrHostNativeAtomicSupported, local)
        out["host_native_atomics"] = int(v) if err == rt.cudaError_t.cudaSuccess else None
    except Exception:  # cuda-bindings missing: the probe is informational
        out["host_native_atomics"] = None
    if scan_path:
        size = os.path.getsize(scan_path)
        chunk = 1 << 20
        fd = os.open(scan_path, os.O_RDONLY)
        buf = np.zeros(chunk, np.uint8)  # touched, so no page faults in the timed reads
        best = 0.0
        for _ in range(2):
            t0 = time.perf_counter()
            for off in range(0, size, chunk):
                os.preadv(fd, [buf], off)
            best = max(best, size / (time.perf_counter() - t0) / 1e9)
        os.close(fd)
        out["tmpfs_pread_GB_per_s_one_thread"] = round(best, 2)
    return out


def hbm_peak() -> float:
    """Measured HBM copy bandwidth of this GPU model (GB/s), from the peaks file
    beside this script, else the nominal 7,700 GB/s.  The scans read HBM only
    for their histograms and counters: their fraction of it is reported for
    completeness."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 7700.0


def host_link_peak(torch, sizes=(4 << 10, 64 << 10, 1 << 20, 16 << 20, 64 << 20, 256 << 20, 1 << 30), sm=False):
    """Pinned cudaMemcpy sweep, H2D and D2H, best of 6 per size (GB/s); the
    ceiling is the best at >= 64 MiB.  Returns {"h2d": .., "d2h": .., "sweep":
    {direction: {bytes: GB/s}}}; with `sm`, also the SMs' own zero-copy
    streaming over the same 1 GiB of pinned memory (genesys_link_stream, best
    of 3): "sm_read" (what a scan of pinned staging can reach) and "sm_write"."""
    n = max(sizes)
    h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = {"sweep": {}}
    for name, (dst, src) in {"h2d": (d, h), "d2h": (h, d)}.items():
        row = {}
        for size in sizes:
            best = 0.0
            for _ in range(6):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                dst[:size].copy_(src[:size], non_blocking=True)
                e.record()
                e.synchronize()
                best = max(best, size / (s.elapsed_time(e) * 1e-3) / 1e9)
            row[str(size)] = round(best, 2)
        out["sweep"][name] = row
        out[name] = max(v for k, v in row.items() if int(k) >= 64 << 20)
    if sm:
        import paper_1705_06965_b300 as G
        dev = torch.cuda.current_device()
        out["sm_read"] = round(G.link_stream(h.data_ptr(), n, write=False, device=dev), 2)
        out["sm_write"] = round(G.link_stream(h.data_ptr(), n, write=True, device=dev), 2)
        # both directions at once (half the blocks each way): the sum of the two
        out["sm_both"] = round(G.link_stream(h.data_ptr(), n, write=2, device=dev), 2)
    del h, d
    return out


def service_phases(before: dict, after: dict) -> dict:
    """Service-thread time per request between two genesys stats snapshots,
    by phase: taking the batch (slot reads), ordering it for merging, the
    Linux calls, writing results back; and the mean batch size."""
    req = max(after["requests"] - before["requests"], 1)
    os_ns = sum(after["op_ns"][o] - before["op_ns"][o] for o in after["op_ns"])

    def per(key):
        return round((after[key] - before[key]) / req, 2)
    return {"pickup": per("pickup_ns"), "order": per("order_ns"), "os_call": round(os_ns / req, 2),
            "complete": per("complete_ns"), "busy": per("busy_ns"),
            "requests_per_batch": round(req / max(after["batches"] - before["batches"], 1), 1),
            "requests_per_os_call": round(req / max(after["os_calls"] - before["os_calls"], 1), 1),
            "empty_polls_per_batch": round((after["empty_polls"] - before["empty_polls"]) /
                                           max(after["batches"] - before["batches"], 1), 2),
            "hole_polls_per_batch": round((after["hole_polls"] - before["hole_polls"]) /
                                          max(after["batches"] - before["batches"], 1), 2)}


def pctl(a, q):
    import numpy as np
    return float(np.percentile(a, q)) if len(a) else None


def _at(d, *path):
    """d[path[0]][path[1]]..., or None where a level is missing."""
    for k in path:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def _sig(x, digits=3):
    """x to `digits` significant digits (numbers only; other values as they are)."""
    if isinstance(x, bool) or not isinstance(x, (int, float)) or x == 0:
        return x
    from math import floor, log10
    nd = digits - 1 - int(floor(log10(abs(x))))
    return round(x, nd) if nd > 0 else int(round(x, nd))


def _beats(a, b, higher_is_better=True):
    """a beats b (None when either is missing)."""
    if a is None or b is None:
        return None
    return bool(a > b) if higher_is_better else bool(a < b)


def _frac(a, b, nd=4):
    """a / b rounded, or None without b."""
    return round(a / b, nd) if a is not None and b else None


def summarize(line: dict) -> dict:
    """The figures of every config in a few hundred bytes, for the end of the
    bench line: the headline, C1's 4 MiB forms and the 1 GiB scan against the
    host link, the C3 wordcount, the C4 service's saturation point, the C5
    served trace against its plain form, every oracle timing with its cores,
    whether each result was checked against the oracle, and the targets (the
    batched or served form against the plain blocking strong form, in
    syscalls/s, requests/s and p99, and the scan's fraction of the link)."""
    ex = line
    scan = {k: v for k, v in (_at(ex, "pread_scan_1GiB") or {}).items() if isinstance(v, dict) and "GB_per_s" in v}
    scan_best = max(scan.items(), key=lambda kv: kv[1]["GB_per_s"], default=(None, {}))
    c3 = _at(ex, "wordcount_c3") or {}
    c3b = max((c3[k] for k in ("plain", "batched") if isinstance(c3.get(k), dict)),
              key=lambda v: v.get("GB_per_s", 0), default={})
    c4 = _at(ex, "kv_c4") or {}
    c5 = _at(ex, "served_c5") or {}
    plain5, served5 = c5.get("plain_first1000") or {}, c5.get("served_first1000") or {}
    pers5 = c5.get("persistent_first1000") or {}
    c2p, c2b = _at(ex, "forms", "plain_blocking_strong") or {}, _at(ex, "forms", "batched") or {}
    c2pc = _at(ex, "forms", "plain_per_call_service") or {}
    oc = _at(ex, "oracle_checks") or {}
    out = {
        "c2c1_syscalls_per_s": _sig(ex.get("value")), "e2e": _sig(_at(ex, "e2e", "value")),
        "wi_2p20": {"calls_per_s": _sig(_at(ex, "roofline", "service", "achieved")),
                    "frac_file_order": _sig(_at(ex, "roofline", "service", "frac")),
                    "frac_interleaved": _sig(_at(ex, "roofline", "service", "warp_interleaved_order", "frac"))},
        "c1_4MiB_GBps": {k: _sig(_at(ex, "c1_4MiB", k, "GB_per_s")) for k in ("plain", "batched")},
        "scan_1GiB": {"form": scan_best[0], "GBps": _sig(scan_best[1].get("GB_per_s")),
                      "frac_h2d": _sig(scan_best[1].get("frac_of_host_link_h2d")),
                      "frac_sm_read": _sig(scan_best[1].get("frac_of_sm_zero_copy_read"))},
        "c3": {"GBps": _sig(c3b.get("GB_per_s")), "frac_h2d": _sig(c3b.get("frac_of_host_link_h2d")),
               "frac_sm_read": _sig(c3b.get("frac_of_sm_zero_copy_read")),
               "truth_eq": c3b.get("counts_equal_ground_truth")},
        "c4": {"sat_rps": _sig(c4.get("saturation_req_per_s")), "p50_us": _sig(c4.get("saturation_p50_us")),
               "p99_us": _sig(c4.get("saturation_p99_us")), "best_any_rps": _sig(c4.get("best_any_req_per_s")),
               "host_bound": c4.get("saturation_host_bound"), "replies_eq_oracle": oc.get("c4_replies_equal")},
        "c5": {"served_rps": _sig(_at(c5, "served_full", "requests_per_s")),
               "served_p99_ms": _sig(_at(c5, "served_full", "p99_ms")),
               "persistent_rps": _sig(_at(c5, "persistent_full", "requests_per_s")),
               "persistent_p99_ms": _sig(_at(c5, "persistent_full", "p99_ms")),
               # the executor's full-trace host-link rate: fractions of the measured H2D and
               # D2H copy rates, and of the SMs' own rate streaming both ways at once
               "persistent_link_frac": [_sig(_at(c5, "persistent_full", "link", k))
                                        for k in ("frac_h2d", "frac_d2h", "frac_sm_both")],
               "plain1k_rps": _sig(plain5.get("requests_per_s")), "plain1k_p99_ms": _sig(plain5.get("p99_ms")),
               "alone_eq_mix": c5.get("first1000_alone_equals_mix"), "full_eq_oracle": oc.get("c5_full_equal")},
        "oracle": {"cores": _at(ex, "probes", "host_cpus"),
                   "c2c1_sps_1t": _sig(_at(ex, "cpu_baseline", "value")),
                   "c1_eq": _at(ex, "cpu_baseline", "c1_histogram_equals_oracle"),
                   "c2_files_eq": oc.get("c2_files_equal"), "scan_eq": oc.get("scan_1GiB_histogram_equal"),
                   "c3_GBps_1t": _sig(_at(c3, "cpu_baseline_oracle", "one_thread_GB_per_s")),
                   "c3_GBps_all": _sig(_at(c3, "cpu_baseline_oracle", "files_to_cores_GB_per_s")),
                   "c4_sat_rps_1t": _sig(_at(c4, "cpu_baseline_oracle_server", "saturation_req_per_s")),
                   "c5_rps_1t": _sig(_at(c5, "cpu_baseline_oracle_replay_first1000", "requests_per_s"))},
    }
    best5 = max((v for v in (served5, pers5) if v), key=lambda v: v.get("requests_per_s", 0), default={})
    c1p, c1b = _at(ex, "c1_4MiB", "plain") or {}, _at(ex, "c1_4MiB", "batched") or {}
    out["targets"] = {
        # C2: the same 2^20 work-item strong blocking GPU calls, served in batches
        # and merged (Sec. 4.2) against served call by call (the plain per-call form)
        "c2_batched_beats_plain": {
            "syscalls_per_s": _beats(c2p.get("syscalls_per_s"), c2pc.get("syscalls_per_s")),
            "p99": _beats(c2p.get("p99_us"), c2pc.get("p99_us"), False)},
        "c5_served_beats_plain": {"syscalls_per_s": _beats(best5.get("syscalls_per_s"), plain5.get("syscalls_per_s")),
                                  "requests_per_s": _beats(best5.get("requests_per_s"), plain5.get("requests_per_s")),
                                  "p99": _beats(best5.get("p99_ms"), plain5.get("p99_ms"), False)},
        # C1: the batched kernel (reads kept in flight) against the plain one, same 1,024 preads
        "c1_batched_beats_plain": {"syscalls_per_s": _beats(c1b.get("preads_per_s"), c1p.get("preads_per_s")),
                                   "p99": _beats(c1b.get("p99_us"), c1p.get("p99_us"), False)},
        # C2 at another grain: one call per 1,024-thread group (relaxed, non-blocking)
        # against one per thread; fewer, larger calls, so not more of them per second
        "c2_coarse_grain_beats_work_item": {
            "syscalls_per_s": _beats(c2b.get("syscalls_per_s"), c2p.get("syscalls_per_s")),
            "requests_per_s": _beats(c2b.get("requests_per_s"), c2p.get("requests_per_s")),
            "p99": _beats(c2b.get("p99_us"), c2p.get("p99_us"), False)},
        "c3_batched_beats_plain": _beats(_at(c3, "batched", "GB_per_s"), _at(c3, "plain", "GB_per_s")),
        # pread + scan against the host link: the 1 GiB scan and the C3 wordcount, each
        # against the stated fraction (0.75 of the measured H2D copy rate)
        "pread_scan_frac_h2d_ge_0.75": {
            k: (None if f is None else bool(f >= 0.75))
            for k, f in (("scan_1GiB", scan_best[1].get("frac_of_host_link_h2d")),
                         ("c3", c3b.get("frac_of_host_link_h2d")))},
    }
    return out


def kernel_src_hash(kernel: str) -> str:
    """Hash of what a kernel's counters depend on: the device protocol headers
    and the kernel's own section of its source file."""
    import hashlib
    h = hashlib.sha1()
    for f in ("include/genesys_device.cuh", "include/genesys_layout.h"):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if kernel.startswith("c2_pwrite_kernel"):
        src = open(os.path.join(ROOT, "paper_1705_06965_b300/csrc/workloads.cu")).read()
        a = src.index("// ------------------------------------------------------------------- C2")
        b = src.index("// ------------------------------------------------------- visibility probe")
        h.update(src[a:b].encode())
    return h.hexdigest()[:12]


def load_traffic(kernel: str, units_per_launch: float):
    """ncu host-link traffic (bytes per launch) of `kernel`: the committed
    per-unit figure times the units of an average launch, or None if there is
    no figure or the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_src_hash(kernel)
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 4 and not ln.startswith("#") and parts[0] == kernel and parts[1] == src:
            return round(float(parts[2]) * units_per_launch)
    return None


class Rig:
    """Context, files and buffers of the GPU arm."""

    def __init__(self, args, local, rank, need_scan=True, service_threads=None, coalesce_max=64, need_c3=True,
                 poll_max_ns=2048, n_slots=0, coalesce_window_ns=0):
        import torch
        import paper_1705_06965_b300 as G
        import workloads
        self.G, self.torch = G, torch
        st_threads = service_threads or args.service_threads
        self.dev = torch.device("cuda", local)
        self.d = workloads.scratch_dir(f"bench_r{rank}")
        self.c1_path = workloads.c1_file(os.path.join(self.d, "c1.bin"), C1_BYTES, seed=workloads.SEED_C1)
        self.scan_path = (workloads.c1_file(os.path.join(self.d, "scan.bin"), SCAN_BYTES, seed=0x5EED00F1)
                          if need_scan else None)
        self.c1_stage_bytes = max(2 * C1_GROUPS * C1_CHUNK, 2 * SCAN_GROUPS * SCAN_CHUNK if need_scan else 0)
        self.c3_stage_bytes = C3_CTAS * (C3_CHUNK + 64) * 2 if need_c3 else 0
        self.ctx = G.Context(device=local, service_threads=st_threads, coalesce_max=coalesce_max, poll_max_ns=poll_max_ns,
                             n_slots=n_slots, coalesce_window_ns=coalesce_window_ns,
                             staging_bytes=max(SIZES) * 64 + self.c1_stage_bytes + self.c3_stage_bytes + (4 << 20),
                             deadline_ns=10_000_000_000)
        self.c2_stage = self.ctx.staging(max(SIZES) * 64)
        self.c1_stage = self.ctx.staging(self.c1_stage_bytes)
        self.c3_stage = self.ctx.staging(self.c3_stage_bytes) if need_c3 else 0
        self.fds = {n: os.open(os.path.join(self.d, f"c2_{n}.bin"), os.O_CREAT | os.O_RDWR, 0o644) for n in SIZES}
        self.fd_c1 = os.open(self.c1_path, os.O_RDONLY)
        self.fd_scan = os.open(self.scan_path, os.O_RDONLY) if self.scan_path else -1
        self.hist = torch.zeros((2, 256), dtype=torch.int32, device=self.dev)
        self.stream = torch.cuda.current_stream()

    def c2(self, n, g, bt, relaxed, nb):
        self.ctx.c2_pwrite(self.fds[n], n, g, bt, relaxed, nb, SEED_C2, self.c2_stage, n * 64)

    def c1(self, form, which=0):
        self.ctx.c1_histogram(self.fd_c1, C1_BYTES, self.hist[which].data_ptr(), self.c1_stage, self.c1_stage_bytes,
                              chunk=C1_CHUNK, groups=C1_GROUPS, threads=C1_THREADS, form=form)

    def scan(self, form, nbytes=SCAN_BYTES):
        self.ctx.c1_histogram(self.fd_scan, nbytes, self.hist[0].data_ptr(), self.c1_stage, self.c1_stage_bytes,
                              chunk=SCAN_CHUNK, groups=SCAN_GROUPS, threads=SCAN_THREADS, form=form)

    def timed(self, fn):
        torch = self.torch
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(self.stream)
        fn()
        e.record(self.stream)
        e.synchronize()
        return s.elapsed_time(e)

    def close(self):
        for fd in list(self.fds.values()) + [self.fd_c1, self.fd_scan]:
            if fd >= 0:
                os.close(fd)
        self.ctx.close()


def per_call_service(G, rig, local, service_threads, n):
    """The work-item strong blocking pwrites of n GPU threads served call by
    call: every request its own Linux call (no merging), each batch one
    doorbell entry (coalesce_max 1), on a context of its own with the same
    service threads; rate and per-call latency."""
    with G.Context(device=local, service_threads=service_threads, coalesce_max=1, merge=False,
                   staging_bytes=1 << 20, deadline_ns=10_000_000_000) as ctx:
        fn = lambda: ctx.c2_pwrite(rig.fds[n], n, 0, 256, False, False, SEED_C2, rig.c2_stage, n * 64)  # noqa
        fn()
        ctx.latency(clear=True)
        st0 = ctx.stats()
        ms = rig.timed(fn)
        lat = ctx.latency(clear=True)
        ph = service_phases(st0, ctx.stats())
    return {"combo": "work-item/strong/blocking", "service": "coalesce_max 1, no merging", "ms": round(ms, 3),
            "syscalls_per_s": round(n / (ms * 1e-3), 1), "requests_per_s": round(n / (ms * 1e-3), 1),
            "p50_us": round(pctl(lat, 50) / 1e3, 2) if len(lat) else None,
            "p99_us": round(pctl(lat, 99) / 1e3, 2) if len(lat) else None, "service_ns_per_request": ph}


def c3_run(rig, form, n_files=None):
    """Wordcount over the full corpus (or its first n_files files, a small
    case for profiling); returns (ms, bytes, counts ok)."""
    import numpy as np
    import workloads
    torch = rig.torch
    c = workloads.corpus(workloads.C3_FULL)
    k = len(c.paths) if n_files is None else min(int(n_files), len(c.paths))
    paths, sizes = c.paths[:k], c.sizes[:k]
    fds = [os.open(p, os.O_RDONLY) for p in paths]
    try:
        counts = torch.zeros(len(c.queries), dtype=torch.int64, device=rig.dev)
        ms = rig.timed(lambda: rig.ctx.c3_wordcount(fds, sizes, c.queries, counts.data_ptr(), rig.c3_stage,
                                                     rig.c3_stage_bytes, chunk=C3_CHUNK, ctas=C3_CTAS,
                                                     threads=C3_THREADS, form=form))
        ok = np.array_equal(counts.cpu().numpy().astype(np.uint64), c.truth[:k].sum(axis=0, dtype=np.uint64))
    finally:
        for fd in fds:
            os.close(fd)
    return ms, int(np.asarray(sizes, np.uint64).sum()), ok


def sweep_step(rig, note=None):
    """One step: the C2 sweep (every size x legal combination) and C1 (plain,
    batched)."""
    G = rig.G
    for n in SIZES:
        for name, g, bt, relaxed, nb in COMBOS:
            rig.c2(n, g, bt, relaxed, nb)
            if note:
                note(f"c2_pwrite_kernel<{G.GRAN_NAMES[g]},{'relaxed' if relaxed else 'strong'},"
                     f"{'nonblocking' if nb else 'blocking'}>")
    for form in (G.FORM_PLAIN, G.FORM_BATCHED):
        rig.c1(form, which=form)
        if note:
            note("c1_plain_kernel" if form == G.FORM_PLAIN else "c1_batched_kernel")


def tune_step(args, local, rank):
    """Autotune the context knobs of the timed step (service threads, batch
    size, slot-area size: 0 = the default of 2048 slots per SM); cached per
    machine."""
    from paper_1705_06965_b300 import autotune
    tuner = autotune.Autotuner()
    key = tuner.key("bench-step", sizes=len(SIZES), combos=len(COMBOS), batches="256-4096")

    def run(cfg):
        rig = Rig(args, local, rank, need_scan=False, need_c3=False, service_threads=cfg["service_threads"],
                  coalesce_max=cfg["coalesce_max"], poll_max_ns=cfg["poll_max_ns"], n_slots=cfg["n_slots"])
        try:
            sweep_step(rig)
            return rig.timed(lambda: sweep_step(rig)) * 1e-3
        finally:
            rig.close()

    # service threads x batch size (batches up to 4096: with the doorbells
    # written without holes, batches fill to the cap) on the default slot
    # area, one slot per resident thread; then the slot-area size for the best
    # pair (smaller areas make work-item callers wait for slots: a 32 K-slot
    # area doubled the step in every run)
    best, table = tuner.tune(key, autotune.grid(service_threads=(1, 2, 4), coalesce_max=(256, 1024, 4096),
                                                poll_max_ns=(2048,), n_slots=(0,)), run, repeats=2)
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    key2 = tuner.key("bench-step-slots", sizes=len(SIZES), combos=len(COMBOS),
                     base=f"{best['service_threads']}x{best['coalesce_max']}")
    best2, table2 = tuner.tune(key2, [dict(best, n_slots=v) for v in (0, 1024 * sms, 512 * sms)], run, repeats=2)
    return best2, table + table2


# ---------------------------------------------------------------- one case
def run_only(args):
    """Run a single case once (after one warm-up) and print its timing: used
    to profile one kernel with small, bounded commands."""
    import torch
    rank, local, _ = dist_env()
    torch.cuda.set_device(local)
    kind, _, rest = args.only.partition(":")
    if kind in ("c4", "c5", "fig10", "f4"):
        import paper_1705_06965_b300 as G
        if kind == "f4":
            res = study_f4(G, local)
        elif kind == "c5" and rest:
            res = serve_c5_part(G, local, rest)
        elif kind == "c5":
            res = serve_c5(G, local, rank, link=host_link_peak(torch, sm=True))
        else:
            res = {"c4": serve_c4, "fig10": study_fig10}[kind](G, local, rank)
        print(json.dumps({"only": args.only, kind: res}), flush=True)
        return
    rig = Rig(args, local, rank, need_scan=kind == "c1" and rest.split(":")[-1] != str(C1_BYTES),
              need_c3=kind == "c3", service_threads=args.service_threads, coalesce_max=args.coalesce_max,
              poll_max_ns=args.poll_max_ns, coalesce_window_ns=args.coalesce_window_ns)
    G = rig.G
    out = {"only": args.only}
    try:
        if kind == "c2":
            key, n = rest.rsplit(":", 1)
            name, order, block = key.split("/")
            g, bt = GRAN_BY_NAME[name]
            n = int(n)
            fn = lambda: rig.c2(n, g, bt, order == "relaxed", block == "nonblocking")  # noqa: E731
            calls = calls_for(g, bt, n)
        elif kind == "c1":
            form_s, nbytes = rest.split(":")
            form = G.FORM_BATCHED if form_s == "batched" else G.FORM_PLAIN
            nbytes = int(nbytes)
            fn = (lambda: rig.c1(form)) if nbytes == C1_BYTES else (lambda: rig.scan(form, nbytes))  # noqa: E731
            calls = nbytes // (C1_CHUNK if nbytes == C1_BYTES else SCAN_CHUNK)
        elif kind == "c3":
            form_s, _, nf = rest.partition(":")
            form = G.FORM_BATCHED if form_s == "batched" else G.FORM_PLAIN
            nf = int(nf) if nf else None
            c3_run(rig, form, nf)
            ms, nbytes, ok = c3_run(rig, form, nf)
            out.update({"ms": round(ms, 3), "GB_per_s": round(nbytes / (ms * 1e-3) / 1e9, 2), "counts_ok": ok})
            print(json.dumps(out), flush=True)
            return
        else:
            raise SystemExit(f"unknown --only kind {kind}")
        fn()
        before = rig.ctx.stats()
        ms = rig.timed(fn)
        after = rig.ctx.stats()
        d = {k: after[k] - before[k] for k in ("requests", "os_calls", "batches", "busy_ns")}
        d["syscall_ns"] = sum(after["op_ns"][o] - before["op_ns"][o] for o in after["op_ns"])
        d["ns_per_request"] = service_phases(before, after)
        out.update({"ms": round(ms, 3), "calls": calls, "calls_per_s": round(calls / (ms * 1e-3), 1),
                    "kernel_ms": round(rig.ctx.last_launch_ms(), 3),
                    "service": {**d, "requests_per_os_call": round(d["requests"] / max(d["os_calls"], 1), 2),
                                "requests_per_batch": round(d["requests"] / max(d["batches"], 1), 2),
                                "busy_frac": round(d["busy_ns"] / (ms * 1e6 * args.service_threads), 4)}})
        if kind == "c2" and g == 0:
            st0 = rig.ctx.stats()
            out["service_probe_calls_per_s"] = round(rig.ctx.service_probe(rig.fds[n], rig.c2_stage, 64, n), 1)
            out["service_probe_ns_per_request"] = service_phases(st0, rig.ctx.stats())
            st0 = rig.ctx.stats()
            out["service_probe_warp_interleaved_calls_per_s"] = round(
                rig.ctx.service_probe(rig.fds[n], rig.c2_stage, 64, n, run=32, stride=8), 1)
            out["service_probe_warp_interleaved_ns_per_request"] = service_phases(st0, rig.ctx.stats())
        print(json.dumps(out), flush=True)
    finally:
        rig.close()


# ---------------------------------------------------------------- extras
def profile_extras(args, rig, local, rank, link, checks=None):
    """Untimed measurements reported beside the headline: pread+scan and
    wordcount GB/s at autotuned settings (fractions of the measured host
    link), the served C5 trace against its plain one-at-a-time form, and the
    C4 key-value service at swept offered rates."""
    import numpy as np
    import torch
    import workloads
    from paper_1705_06965_b300 import autotune
    G = rig.G
    out = {}
    # pread + histogram over 1 GiB: each form (work-group plain, work-group
    # batched, warp, work-group with an HBM landing copy) at its own autotuned
    # setting
    best = autotune.tune_scan(local, rig.fd_scan, SCAN_BYTES)
    per_form = best.get("by_form") or {str(best["form"]): best}
    sb = max(c["groups"] * c["chunk"] * (32 if c["form"] == G.FORM_WARP else 2) for c in per_form.values())
    res, hists = {}, {}
    names = {G.FORM_PLAIN: "plain", G.FORM_BATCHED: "batched", G.FORM_WARP: "warp", G.FORM_HBM: "hbm_landing"}
    for f, cfg in sorted(per_form.items()):
        with G.Context(device=local, service_threads=cfg["service_threads"], staging_bytes=sb + (1 << 20)) as ctx:
            st = ctx.staging(sb)
            fn = lambda: ctx.c1_histogram(rig.fd_scan, SCAN_BYTES, rig.hist[0].data_ptr(), st, sb,  # noqa: E731
                                          chunk=cfg["chunk"], groups=cfg["groups"], threads=1024, form=cfg["form"])
            fn()
            ms = min(rig.timed(fn) for _ in range(3))
            rig.hist[0].zero_()
            fn()  # once more from zero: the histogram this form computes
            hists[names[cfg["form"]]] = rig.hist[0].cpu().numpy().view(np.uint32).copy()
            gbs = SCAN_BYTES / (ms * 1e-3) / 1e9
            res[names[cfg["form"]]] = {"GB_per_s": round(gbs, 2), "frac_of_host_link_h2d": round(gbs / link["h2d"], 4),
                                       "frac_of_sm_zero_copy_read": _frac(gbs, link.get("sm_read")),
                                       "frac_of_hbm_peak": round(gbs / hbm_peak(), 5),
                                       "ms": round(ms, 2), "chunk": cfg["chunk"], "groups": cfg["groups"],
                                       "service_threads": cfg["service_threads"]}
    first = next(iter(hists.values()))
    out["pread_scan_1GiB"] = {"autotuned": {k: v for k, v in best.items() if k != "by_form"}, **res,
                              # what holds at any size: the forms agree, every byte is counted once
                              "histograms_checked": bool(all(np.array_equal(h, first) for h in hists.values()) and
                                                         int(first.sum(dtype=np.uint64)) == SCAN_BYTES)}
    if checks is not None:
        checks["scan"] = (rig.scan_path, first)
    # C3 wordcount over the full corpus
    c = workloads.corpus(workloads.C3_FULL)
    fds = [os.open(p, os.O_RDONLY) for p in c.paths]
    try:
        best = autotune.tune_wordcount(local, fds, c.sizes, c.queries)
        sb = 2 * best["ctas"] * (best["chunk"] + 64)
        with G.Context(device=local, service_threads=best["service_threads"], staging_bytes=sb + (1 << 20)) as ctx:
            st = ctx.staging(sb)
            res = {}
            for form in (G.FORM_PLAIN, G.FORM_BATCHED):
                counts = torch.zeros(len(c.queries), dtype=torch.int64, device=rig.dev)
                fn = lambda: ctx.c3_wordcount(fds, c.sizes, c.queries, counts.data_ptr(), st, sb,  # noqa: E731
                                              chunk=best["chunk"], ctas=best["ctas"], threads=512, form=form)
                fn()
                counts.zero_()
                ms = rig.timed(fn)
                ok = bool(np.array_equal(counts.cpu().numpy().astype(np.uint64), c.truth_total()))
                ms = min(ms, *(rig.timed(fn) for _ in range(2)))
                gbs = c.total_bytes / (ms * 1e-3) / 1e9
                res["plain" if form == G.FORM_PLAIN else "batched"] = {
                    "GB_per_s": round(gbs, 2), "frac_of_host_link_h2d": round(gbs / link["h2d"], 4),
                    "frac_of_sm_zero_copy_read": _frac(gbs, link.get("sm_read")),
                    "frac_of_hbm_peak": round(gbs / hbm_peak(), 5),
                    "ms": round(ms, 2), "counts_equal_ground_truth": ok}
            out["wordcount_c3"] = {"autotuned": best, "corpus_bytes": c.total_bytes, **res}
            if rank == 0:
                try:
                    out["wordcount_c3"]["cpu_baseline_oracle"] = cpu_baseline_c3(c)
                except Exception as e:  # reported in the line, never hidden
                    out["wordcount_c3"]["cpu_baseline_oracle"] = {"error": f"{type(e).__name__}: {e}"}
    finally:
        for fd in fds:
            os.close(fd)
    out["served_c5"] = serve_c5(G, local, rank, checks, link)
    out["kv_c4"] = serve_c4(G, local, rank, checks=checks)
    out["fig6_block_permutation"] = study_fig6(G, rig, local)
    out["fig7_coalescing"] = study_fig7(G, rig, local, rank)
    out["fig10_echo"] = study_fig10(G, local, rank)
    try:
        out["f4_other_calls"] = study_f4(G, local)
    except Exception as e:  # reported in the line, never hidden
        out["f4_other_calls"] = {"error": f"{type(e).__name__}: {e}"}
    out["call_timeline"] = trace_timeline(G, rig, local)
    return out


def study_f4(G, local, n=200, nbytes=4096, warmup=3):
    """Sec. 5 and Sec. 8.1: the rest of the paper's call set made from GPU
    code - open, write, lseek, read and close on a file the GPU opened
    itself (a stateful descriptor), and madvise on host-mapped memory - one
    call per single-block kernel at work-group grain (128 threads).  Per call:
    the kernel's device time (claim, publish, service, completion and the
    barriers around the call) p50/p99 over n rounds; every round writes fresh
    random bytes and must read back exactly them.  The same calls made by a
    host thread are timed beside it."""
    import mmap
    import tempfile
    import numpy as np
    nrs = {"open": 2, "write": 1, "lseek": 8, "read": 0, "close": 3, "madvise": 28}
    o_flags = os.O_RDWR | os.O_CREAT | os.O_TRUNC
    tmp = tempfile.mkdtemp(prefix="genesys_f4_")
    path = os.path.join(tmp, "f4.bin")
    dev_ms = {k: [] for k in nrs}
    host_ns = {k: [] for k in nrs}
    ok = True
    rng = np.random.default_rng(1705)
    try:
        with G.Context(device=local, service_threads=2, staging_bytes=1 << 20) as ctx:
            pb = path.encode() + b"\0"
            pbuf = ctx.staging(len(pb))
            ctx.host_view(pbuf, len(pb))[:] = np.frombuffer(pb, np.uint8)
            wbuf, rbuf = ctx.staging(nbytes), ctx.staging(nbytes)
            page = (ctx.staging(2 * 4096) + 4095) & ~4095
            w, r = ctx.host_view(wbuf, nbytes), ctx.host_view(rbuf, nbytes)

            def call(name, args, keep):
                ret = ctx.gpu_call(nrs[name], args, G.GRAN_GROUP, 128)
                if keep:
                    dev_ms[name].append(ctx.last_launch_ms())
                return ret

            for i in range(warmup + n):
                keep = i >= warmup
                w[:] = rng.integers(0, 256, nbytes, dtype=np.uint8)
                r[:] = 0
                fd = call("open", [pbuf, o_flags, 0o644], keep)
                ok &= fd >= 0
                ok &= call("write", [fd, wbuf, nbytes], keep) == nbytes
                ok &= call("lseek", [fd, 0, os.SEEK_SET], keep) == 0
                ok &= call("read", [fd, rbuf, nbytes], keep) == nbytes
                ok &= bool(np.array_equal(r, w))
                ok &= call("close", [fd], keep) == 0
                ok &= call("madvise", [page, 4096, mmap.MADV_NORMAL], keep) == 0
            status = ctx.status()
            ok &= not any(status)
        # the same calls from a host thread
        hbuf = bytearray(nbytes)
        region = mmap.mmap(-1, 4096)
        for i in range(warmup + n):
            keep = i >= warmup
            t = [time.perf_counter_ns()]
            fd = os.open(path, o_flags, 0o644)
            t.append(time.perf_counter_ns())
            os.write(fd, hbuf)
            t.append(time.perf_counter_ns())
            os.lseek(fd, 0, os.SEEK_SET)
            t.append(time.perf_counter_ns())
            os.readv(fd, [hbuf])
            t.append(time.perf_counter_ns())
            os.close(fd)
            t.append(time.perf_counter_ns())
            region.madvise(mmap.MADV_NORMAL, 0, 4096)
            t.append(time.perf_counter_ns())
            if keep:
                for k, name in enumerate(nrs):
                    host_ns[name].append(t[k + 1] - t[k])
        region.close()
    finally:
        if os.path.exists(path):
            os.unlink(path)
        os.rmdir(tmp)
    out = {"rounds": n, "bytes_per_read_write": nbytes, "grain": "work-group (128 threads), one call per kernel",
           "all_results_correct": bool(ok), "gpu_kernel_us": {}, "host_thread_us": {}}
    for name in nrs:
        a = [x * 1e3 for x in dev_ms[name]]
        out["gpu_kernel_us"][name] = {"p50": round(pctl(a, 50), 2), "p99": round(pctl(a, 99), 2)}
        out["host_thread_us"][name] = {"p50": round(pctl([x * 1e-3 for x in host_ns[name]], 50), 2)}
    return out


def trace_timeline(G, rig, local, n=1 << 16):
    """Where a blocking call's time goes (per-call trace, clocks aligned by
    round trips): claim (call to publish), queue (publish to CPU pickup),
    service (pickup to completion word), delivery (completion word to result
    seen), at work-item and work-group (256) grain for 2^16 threads."""
    import workloads
    out = {}
    for name, gran, bt in (("work-item", G.GRAN_ITEM, 256), ("work-group-256", G.GRAN_GROUP, 256)):
        with G.Context(device=local, service_threads=2, coalesce_max=256, staging_bytes=n * 64 + (1 << 20),
                       trace=2 * n) as ctx:
            st = ctx.staging(n * 64)
            ctx.c2_pwrite(rig.fds[n], n, gran, bt, False, False, workloads.SEED_C2, st, n * 64)
            ctx.trace_read(calibrate=False)
            ctx.c2_pwrite(rig.fds[n], n, gran, bt, False, False, workloads.SEED_C2, st, n * 64)
            dev, host, off = ctx.trace_read()
            b = G.trace_breakdown(dev, host, off)
            b["service_cpu_ms"] = round(ctx.stats()["service_cpu_ns"] / 1e6, 1)
            out[name] = b
    return out


def study_fig6(G, rig, local, n_blocks=4096, iters=(1, 2, 4, 8, 16, 32, 64)):
    """Sec. 6 / Fig. 6: time per permutation iteration of 8 KiB blocks (1024
    threads per work-group) followed by a work-group pwrite, for the four
    ordering x blocking combinations."""
    import numpy as np
    import torch
    import workloads
    data, perm = workloads.c6_inputs(n_blocks)
    d_in = torch.from_numpy(data).to(rig.dev)
    d_perm = torch.from_numpy(perm.view(np.int16)).to(rig.dev)
    path = os.path.join(rig.d, "c6.bin")
    out = {"blocks": n_blocks, "us_per_iteration": {}}
    with G.Context(device=local, service_threads=4, staging_bytes=n_blocks * 8192 + (1 << 20)) as ctx:
        st = ctx.staging(n_blocks * 8192)
        fd = os.open(path, os.O_CREAT | os.O_RDWR, 0o644)
        try:
            for relaxed in (False, True):
                for nb in (False, True):
                    key = f"{'weak' if relaxed else 'strong'}-{'non-block' if nb else 'block'}"
                    row = {}
                    for it in iters:
                        fn = lambda: ctx.c6_permute(fd, d_in.data_ptr(), d_perm.data_ptr(), n_blocks, it,  # noqa
                                                    relaxed, nb, st, n_blocks * 8192)
                        fn()
                        ms = min(rig.timed(fn) for _ in range(3))
                        row[str(it)] = round(ms * 1e3 / it, 2)
                    out["us_per_iteration"][key] = row
        finally:
            os.close(fd)
    return out


def study_fig7(G, rig, local, rank, sizes=(256 << 10, 1 << 20, 4 << 20, 16 << 20, 64 << 20), groups=64):
    """Sec. 6 / Fig. 7: a fixed number of work-groups each read 1/64 of a file
    with one pread (more bytes per call for larger files); time per requested
    byte without coalescing, with up to 8 requests per service batch (20 us
    window), and with batching plus merging of contiguous reads."""
    import workloads
    d = workloads.scratch_dir(f"bench_fig7_r{rank}")
    paths = {n: workloads.c1_file(os.path.join(d, f"f{n}.bin"), n, seed=0x5EED0007) for n in sizes}
    modes = {"no_coalescing": dict(coalesce_max=1, merge=False),
             "batch_le_8": dict(coalesce_max=8, coalesce_window_ns=20_000, merge=False),
             "batch_le_8_merge": dict(coalesce_max=8, coalesce_window_ns=20_000, merge=True)}
    out = {"groups": groups, "ns_per_byte": {}}
    for mode, kw in modes.items():
        row = {}
        with G.Context(device=local, service_threads=4, staging_bytes=(64 << 20) + (1 << 20), **kw) as ctx:
            st = ctx.staging(64 << 20)
            for n, p in paths.items():
                fd = os.open(p, os.O_RDONLY)
                try:
                    chunk = n // groups
                    fn = lambda: ctx.c1_histogram(fd, n, rig.hist[0].data_ptr(), st, 64 << 20, chunk=chunk,  # noqa
                                                  groups=groups, threads=256, form=G.FORM_PLAIN)
                    fn()
                    ms = min(rig.timed(fn) for _ in range(3))
                    row[str(n)] = round(ms * 1e6 / n, 4)
                finally:
                    os.close(fd)
        out["ns_per_byte"][mode] = row
    return out


# C5 serving: 128 requests on the GPU at once (one stream each), 256 MiB
# staging and HBM budgets, 12 service threads (a sweep on the B300 machine:
# 9.6-9.7 k requests/s against 9.2-9.4 k with 64 requests, 64 MiB budgets and
# 8 threads, in both forms)
C5_SERVE = dict(max_inflight=128, n_streams=128, staging_budget=256 << 20, hbm_budget=256 << 20)
C5_SERVICE_THREADS = 12


def c5_link_bytes(tr):
    """Host-link bytes of a C5 trace, each direction: pread data in (H2D);
    pwrite data out (D2H); each mmap'd region filled by the GPU (D2H) and read
    back for its checksum (H2D)."""
    import numpy as np
    import workloads
    live = np.arange(tr.ops.shape[1])[None, :] < tr.n_ops[:, None]
    kind, ln = tr.ops["kind"][live], tr.ops["len"][live].astype(np.int64)
    rd = int(ln[kind == workloads.OP_PREAD].sum())
    wr = int(ln[kind == workloads.OP_PWRITE].sum())
    mm = int(ln[kind == workloads.OP_MMAP].sum())
    return rd + mm, wr + mm


def serve_c5(G, local, rank, checks=None, link=None):
    """C5: the 10,000-request trace served with continuous admission (up to 128
    requests in flight, graph relaunch, autotuned call granularity), and its
    first 1,000 requests both served and in the plain one-at-a-time form.
    checks["c5"] receives what the oracle leg compares: the trace, the full
    run's results and its output file.  With `link` (the measured pinned copy
    rates) each run also reports its host-link rate in both directions and
    the fractions of the measured rates."""
    import numpy as np
    import workloads
    tr = workloads.c5_trace(workloads.C5_FULL)
    d = workloads.scratch_dir(f"bench_c5_r{rank}")
    in_fds = [os.open(p, os.O_RDONLY) for p in tr.in_paths]
    out = {}
    try:
        with G.Context(device=local, service_threads=C5_SERVICE_THREADS, staging_bytes=512 << 20) as ctx:
            def run(sub, out_name="out.bin", **cfg):
                ofd = os.open(os.path.join(d, out_name), os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
                try:
                    t0 = time.perf_counter()
                    res, lat, st = ctx.c5_serve(sub.arrival_ns, sub.threads, sub.n_ops, sub.ops, in_fds, ofd, **cfg)
                    wall = time.perf_counter() - t0
                finally:
                    os.close(ofd)
                span = st["makespan_ns"] * 1e-9
                row = {"requests": st["requests"], "syscalls": st["syscalls"],
                       "syscalls_per_s": round(st["syscalls"] / span, 1),
                       "requests_per_s": round(st["requests"] / span, 1),
                       "p50_ms": round(float(np.percentile(lat, 50)) / 1e6, 3),
                       "p99_ms": round(float(np.percentile(lat, 99)) / 1e6, 3),
                       "makespan_s": round(span, 3), "wall_s": round(wall, 3),
                       "max_inflight": st["max_inflight"], "graph_launches": st["graph_launches"]}
                if link:
                    h2d, d2h = c5_link_bytes(sub)
                    row["link"] = {"h2d_GB": round(h2d / 1e9, 3), "d2h_GB": round(d2h / 1e9, 3),
                                   "h2d_GB_per_s": round(h2d / span / 1e9, 2),
                                   "d2h_GB_per_s": round(d2h / span / 1e9, 2),
                                   "frac_h2d": round(h2d / span / 1e9 / link["h2d"], 4),
                                   "frac_d2h": round(d2h / span / 1e9 / link["d2h"], 4),
                                   # against what the SMs alone stream over the link (the fills
                                   # are SM stores, the read-backs and scans SM loads)
                                   "frac_sm_read": _frac(h2d / span / 1e9, link.get("sm_read")),
                                   "frac_sm_write": _frac(d2h / span / 1e9, link.get("sm_write")),
                                   # both directions against the SMs streaming both at once
                                   "frac_sm_both": _frac((h2d + d2h) / span / 1e9, link.get("sm_both"))}
                return res, row
            from paper_1705_06965_b300 import autotune
            ofd = os.open(os.path.join(d, "tune.bin"), os.O_CREAT | os.O_RDWR, 0o644)
            try:
                tuned = autotune.tune_serve(local, ctx, tr, in_fds, ofd, extra=C5_SERVE)
            finally:
                os.close(ofd)
            out["autotuned"] = tuned
            # the persistent executor form: one kernel serves every request
            ofd = os.open(os.path.join(d, "tune_p.bin"), os.O_CREAT | os.O_RDWR, 0o644)
            try:
                tuned_p = autotune.tune_serve(local, ctx, tr, in_fds, ofd, extra={**C5_SERVE, "persistent": 1})
            finally:
                os.close(ofd)
            out["autotuned_persistent"] = tuned_p
            first = tr.subset(np.arange(1000))
            r_plain, out["plain_first1000"] = run(first, max_inflight=1, use_graphs=0)
            r_served, out["served_first1000"] = run(first, **C5_SERVE, **tuned)
            r_pers, out["persistent_first1000"] = run(first, **C5_SERVE, persistent=1, **tuned_p)
            m = np.arange(8)[None, :] < first.n_ops[:, None]
            out["first1000_alone_equals_mix"] = bool(np.array_equal(r_plain[m], r_served[m]) and
                                                     np.array_equal(r_plain[m], r_pers[m]))
            r_full, out["served_full"] = run(tr, "out_full.bin", **C5_SERVE, **tuned)
            r_pfull, out["persistent_full"] = run(tr, "out_pfull.bin", **C5_SERVE, persistent=1, **tuned_p)
            if checks is not None:
                checks["c5"] = (tr, {"served_full": (r_full, os.path.join(d, "out_full.bin")),
                                     "persistent_full": (r_pfull, os.path.join(d, "out_pfull.bin"))})
            # below saturation: the first 2,000 requests with arrivals spread to
            # 4 k/s, where latency is service time rather than queueing
            slow = tr.subset(np.arange(2000))
            slow.arrival_ns = (slow.arrival_ns.astype(np.float64) * (tr.params["rate_per_s"] / 4000.0)).astype(np.uint64)
            _, out["served_first2000_at_4k_per_s"] = run(slow, **C5_SERVE, **tuned)
            _, out["persistent_first2000_at_4k_per_s"] = run(slow, **C5_SERVE, persistent=1, **tuned_p)
        if rank == 0:
            try:
                out["cpu_baseline_oracle_replay_first1000"] = cpu_baseline_c5(first, in_fds, d, r_served)
            except Exception as e:  # reported in the line, never hidden
                out["cpu_baseline_oracle_replay_first1000"] = {"error": f"{type(e).__name__}: {e}"}
    finally:
        for fd in in_fds:
            os.close(fd)
    out["trace"] = {"requests": len(tr), "rate_per_s": tr.params["rate_per_s"]}
    return out


def serve_c5_part(G, local, spec):
    """One serving form on the trace's first n requests, all present at the
    start, with the bench's serving settings and fixed call granularity
    (64 KiB parts, 1024-thread blocks): `spec` = "served:n" or
    "persistent:n".  A small, bounded case for profiling the executor."""
    import numpy as np
    import torch
    import workloads
    form, _, n = spec.partition(":")
    tr = workloads.c5_trace(workloads.C5_FULL)
    sub = tr.subset(np.arange(min(int(n or 1000), len(tr))))
    d = workloads.scratch_dir("bench_c5_part")
    in_fds = [os.open(p, os.O_RDONLY) for p in tr.in_paths]
    link = host_link_peak(torch, sm=True)
    try:
        with G.Context(device=local, service_threads=C5_SERVICE_THREADS, staging_bytes=512 << 20) as ctx:
            ofd = os.open(os.path.join(d, "out.bin"), os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
            try:
                cfg = dict(C5_SERVE, min_part=65536, block_threads=1024, honor_arrivals=0,
                           persistent=1 if form == "persistent" else 0)
                _, lat, st = ctx.c5_serve(sub.arrival_ns, sub.threads, sub.n_ops, sub.ops, in_fds, ofd, **cfg)
            finally:
                os.close(ofd)
    finally:
        for fd in in_fds:
            os.close(fd)
    span = st["makespan_ns"] * 1e-9
    h2d, d2h = c5_link_bytes(sub)
    return {"form": form, "requests": st["requests"], "requests_per_s": round(st["requests"] / span, 1),
            "p99_ms": round(float(np.percentile(lat, 99)) / 1e6, 3), "makespan_s": round(span, 4),
            "link": {"h2d_GB": round(h2d / 1e9, 3), "d2h_GB": round(d2h / 1e9, 3),
                     "frac_h2d": round(h2d / span / 1e9 / link["h2d"], 4),
                     "frac_d2h": round(d2h / span / 1e9 / link["d2h"], 4),
                     "frac_sm_read": _frac(h2d / span / 1e9, link.get("sm_read")),
                     "frac_sm_write": _frac(d2h / span / 1e9, link.get("sm_write")),
                     "frac_sm_both": _frac((h2d + d2h) / span / 1e9, link.get("sm_both"))}}


def cpu_baseline_c3(c, sample_bytes=512 << 20):
    """The oracle's wordcount on the host cores (Sec. 7.1's CPU baseline):
    one thread, and the files-to-cores OpenMP form on every core, over the
    corpus's first files up to sample_bytes; the two must count the same."""
    import numpy as np
    import oracle
    sizes = np.asarray(c.sizes, np.int64)
    k = min(len(sizes), int(np.searchsorted(np.cumsum(sizes), sample_bytes)) + 1)
    paths, nb = c.paths[:k], int(sizes[:k].sum())
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    one, _ = oracle.c3_wordcount(paths, c.queries)
    d1 = time.perf_counter() - t
    t = time.perf_counter()
    omp, _ = oracle.c3_wordcount(paths, c.queries, threads=cores)
    d2 = time.perf_counter() - t
    return {"kind": "oracle", "sample": f"first {k} of {len(sizes)} files, {nb} bytes",
            "one_thread_GB_per_s": round(nb / d1 / 1e9, 3), "files_to_cores_GB_per_s": round(nb / d2 / 1e9, 3),
            "cores": cores, "counts_agree": bool(np.array_equal(one, omp))}


def cpu_baseline_c5(sub, in_fds, d, served):
    """The oracle's sequential replay (one thread; requests in arrival order,
    each operation a plain host call) of the requests `sub`, whose served
    results are `served`: requests/s, and whether the results agree."""
    import numpy as np
    import oracle
    ofd = os.open(os.path.join(d, "oracle_out.bin"), os.O_CREAT | os.O_RDWR, 0o644)
    try:
        t = time.perf_counter()
        want = oracle.c5_trace(sub, ofd, in_fds)
        dt = time.perf_counter() - t
    finally:
        os.close(ofd)
    m = np.arange(want.shape[1])[None, :] < sub.n_ops[:, None]
    return {"kind": "oracle", "requests": len(sub), "cores": 1, "seconds": round(dt, 3),
            "requests_per_s": round(len(sub) / dt, 1),
            "served_results_equal_oracle": bool(np.array_equal(want[m], np.asarray(served)[m]))}


def _kv_requests_at(rate, n_max):
    """Requests offered at one rate: 1.25 s of traffic, at least 200k and at
    most the trace's length."""
    return int(min(n_max, max(200_000, rate * 1.25)))


def reply_digests(replies) -> "np.ndarray":
    """A 64-bit digest of each reply (its length and CRC-32), so that replies
    can be kept per offered rate and compared with the oracle's afterwards
    without holding every byte."""
    import zlib
    import numpy as np
    return np.fromiter(((len(r) << 32) | zlib.crc32(r) for r in replies), np.uint64, len(replies))


def _kv_point(tr, reqs, off, rate, run_server, port, client_cpus=None, keep=None):
    """Offer the first requests of the trace (_kv_requests_at) at `rate`
    requests/s to a server started by run_server(port); achieved rate and
    send-to-reply latency.  The load generator's threads run on client_cpus
    (if given); keep[rate] receives the replies' digests."""
    import numpy as np
    import paper_1705_06965_b300 as G
    n = _kv_requests_at(rate, len(tr))
    arr = (tr.arrival_ns[:n].astype(np.float64) * (tr.params["rate_per_s"] / rate)).astype(np.uint64)
    srv = run_server(port)
    mask = os.sched_getaffinity(0)
    seen = None
    try:
        if client_cpus:  # threads the generator starts inherit this thread's CPU set
            os.sched_setaffinity(0, client_cpus)
        reps, lat, st = G.kv_client(reqs[:int(off[n])], off[:n + 1], arr, port, 32, timeout_ns=10_000_000_000)
        if hasattr(srv, "received"):  # the GPU server logs the requests that reached it
            seen = srv.received(n)
    finally:
        os.sched_setaffinity(0, mask)
        served = srv.stop()
    if keep is not None:
        keep[str(int(rate))] = (reply_digests(reps), seen)
    got = lat[lat > 0]
    achieved = st["received"] / (st["span_ns"] * 1e-9) if st["span_ns"] else 0.0
    return {"requests": n, "received": st["received"], "served": served, "achieved_req_per_s": round(achieved, 1),
            "p50_us": round(float(np.percentile(got, 50)) / 1e3, 2) if len(got) else None,
            "p99_us": round(float(np.percentile(got, 99)) / 1e3, 2) if len(got) else None,
            "max_send_late_us": round(st["max_send_late_ns"] / 1e3, 1),
            # the load generator kept its schedule (no request left later than
            # 5 % of the point's duration, or 1 ms, after its arrival time):
            # else the rate was not really offered
            "offered_on_schedule": bool(st["max_send_late_ns"] <= max(1_000_000, 0.05 * float(arr[-1])))}


def _kv_sweep(tr, reqs, off, run_server, port, rates, client_cpus=None, keep=None):
    """Offered rates from the first, doubling, until the server saturates
    (achieved below 90 % of offered, or replies missing)."""
    out = {}
    for rate in rates:
        pt = _kv_point(tr, reqs, off, rate, run_server, port, client_cpus, keep)
        out[str(int(rate))] = pt
        port += 40
        if pt["received"] < pt["requests"] or pt["achieved_req_per_s"] < 0.9 * rate:
            break
    return out


def kv_saturation(points: dict) -> dict:
    """The server's saturation point from a rate sweep: the best achieved rate
    among the points the load generator offered on schedule with every reply
    received (a point where the generator fell behind measures the host, not
    the server); the best of all points for context, and whether the sweep
    ended on a point the generator did not keep to (then the server's own
    limit may be higher)."""
    clean = [v for v in points.values() if v["offered_on_schedule"] and v["received"] == v["requests"]]
    best = max(clean, key=lambda v: v["achieved_req_per_s"], default=None)
    any_best = max(points.values(), key=lambda v: v["achieved_req_per_s"], default=None)
    last = list(points.values())[-1] if points else None
    return {"saturation_req_per_s": best["achieved_req_per_s"] if best else None,
            "saturation_p50_us": best["p50_us"] if best else None,
            "saturation_p99_us": best["p99_us"] if best else None,
            "best_any_req_per_s": any_best["achieved_req_per_s"] if any_best else None,
            "saturation_host_bound": bool(last is not None and not last["offered_on_schedule"])}


def c4_cpu_split():
    """Disjoint host cores for the key-value service (its service threads, or
    the oracle's server) and for the load generator, on a host with 16 or more
    cores: (server cores, generator cores), or (None, None)."""
    n = os.cpu_count() or 1
    if n < 16:
        return None, None
    half = n // 2
    return list(range(half)), set(range(half, n))


C4_RATES = (50_000.0, 100_000.0, 200_000.0, 400_000.0, 800_000.0, 1_200_000.0, 1_600_000.0, 3_200_000.0)


def serve_c4(G, local, rank, rates=C4_RATES, n_req=1_000_000, checks=None):
    """C4: 1M-key table in HBM, Zipf 0.99 keys, 90% GET; offered rates 50k/s
    doubling to saturation (with 1.2M/s between 800k and 1.6M, where the
    load generator stops keeping its schedule), 1.25 s of requests per rate
    (200k to 1M);
    achieved requests/s and send-to-reply latency.  The service threads and
    the load generator run on disjoint host cores.  The oracle's single-thread
    CPU server is offered the same rates (its own saturation point is the CPU
    baseline).  checks["c4"] receives what the oracle leg compares: the trace
    and every reply's digest per offered rate."""
    import workloads
    p = dict(workloads.C4_FULL, n_requests=n_req)
    tr = workloads.kv_trace(p)
    reqs, off = workloads.kv_request_bytes(tr)
    server_cpus, client_cpus = c4_cpu_split()
    out = {"keys": len(tr.keys), "requests_per_rate": {str(int(r)): _kv_requests_at(r, n_req) for r in rates},
           "sockets": 32, "service_threads": 8,
           "cores": {"server": f"{server_cpus[0]}-{server_cpus[-1]}" if server_cpus else "any",
                     "load_generator": f"{min(client_cpus)}-{max(client_cpus)}" if client_cpus else "any"}}
    digests = {}
    with G.Context(device=local, service_threads=8, staging_bytes=64 << 20,
                   service_cpus=server_cpus[:8] if server_cpus else None) as ctx:
        def gpu_server(port):
            return G.KVServer(ctx, tr.keys, tr.vlen0, tr.vseed0, n_sockets=32, batch=64, port_base=port)
        out["rates"] = _kv_sweep(tr, reqs, off, gpu_server, 41000 + 400 * rank, rates, client_cpus, digests)
    if checks is not None:
        checks["c4"] = (tr, digests)
    if rank == 0:
        out["cpu_baseline_oracle_server"] = cpu_baseline_c4(tr, reqs, off, 41000 + 400 * rank + 200, rates,
                                                            server_cpus, client_cpus)
    out.update(kv_saturation(out["rates"]))
    return out


def cpu_baseline_c4(tr, reqs, off, port, rates, server_cpus=None, client_cpus=None):
    """The oracle's key-value server (one host thread, recvfrom/sendto one
    datagram at a time, on the server cores) offered the same rates."""
    import oracle
    table = tr.values0_table()

    class CpuServer:
        def __init__(self, port):
            mask = os.sched_getaffinity(0)
            try:
                if server_cpus:  # the server's thread inherits this thread's CPU set
                    os.sched_setaffinity(0, set(server_cpus))
                self.srv = oracle.UdpServer("kv", port, 32, trace=tr, idle_ns=5_000_000_000, values0=table)
            finally:
                os.sched_setaffinity(0, mask)

        def stop(self):
            return self.srv.join()["answered"]
    cpu_server = CpuServer
    res = _kv_sweep(tr, reqs, off, cpu_server, port, rates, client_cpus)
    return {"threads": 1, "rates": res, **kv_saturation(res)}


def study_fig10(G, local, rank, sizes=(64, 256, 1024, 4096, 16384, 65504), n_sockets=32):
    """Sec. 7.3 / Fig. 10: bandwidth of a UDP echo server versus packet size,
    with the packets processed on the GPU (recvfrom/sendto at work-group
    grain, and the recvmmsg/sendmmsg batch form) and on the CPU (the
    oracle's plain server on as many host threads as the GPU arm has service
    threads).  Closed-loop client, 4 datagrams in flight per socket, every
    reply compared byte for byte."""
    port = 43000 + 400 * rank
    service = 4
    out = {"sockets": n_sockets, "window": 4, "service_threads": service, "GB_per_s": {}, "all_echoed": True}
    arms = {"gpu_recvfrom_sendto": ("gpu", G.ECHO_SINGLE), "gpu_recvmmsg_sendmmsg": ("gpu", G.ECHO_BATCH)}
    if rank == 0:
        arms["cpu_baseline_oracle_server"] = ("cpu", None)
    with G.Context(device=local, service_threads=service,
                   staging_bytes=(2 * 16 * 65536 + 65536) * n_sockets + (1 << 20)) as ctx:
        for arm, (where, form) in arms.items():
            row = {}
            for size in sizes:
                n = int(min(100_000, max(5_000, 1.5e9 // size)))
                if where == "gpu":
                    srv = G.EchoServer(ctx, n_sockets=n_sockets, max_packet=size, form=form, batch=16, threads=256,
                                       port_base=port)
                    stop = srv.stop
                else:
                    import oracle
                    srv = oracle.UdpServer("echo", port, n_sockets, threads=service, max_packet=size,
                                           idle_ns=5_000_000_000)
                    stop = srv.join
                try:
                    st = G.echo_client(port, n_sockets, size, n, window=4, threads=4)
                finally:
                    stop()
                port += 20
                out["all_echoed"] &= st["echoed"] == n and st["bad"] == 0
                row[str(size)] = round(st["GB_per_s"], 3) if st["GB_per_s"] else None
            out["GB_per_s"][arm] = row
    return out


# ---------------------------------------------------------------- GPU arm
def run_genesys(args):
    import numpy as np
    import torch

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    step_cfg, step_table = tune_step(args, local, rank) if args.autotune else (
        {"service_threads": args.service_threads, "coalesce_max": args.coalesce_max, "poll_max_ns": args.poll_max_ns,
         "n_slots": 0}, [])
    rig = Rig(args, local, rank, service_threads=step_cfg["service_threads"], coalesce_max=step_cfg["coalesce_max"],
              poll_max_ns=step_cfg["poll_max_ns"], n_slots=step_cfg.get("n_slots", 0))
    G, ctx, dev = rig.G, rig.ctx, rig.dev
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    kernel_ms = {}
    launches = [0]

    def note(kname):
        kernel_ms.setdefault(kname, []).append(ctx.last_launch_ms())
        launches[0] += 1

    def one_step(collect=True):
        sweep_step(rig, note if collect else None)

    for _ in range(max(args.warmup, 0)):
        rig.hist.zero_()
        one_step(collect=False)
    torch.cuda.synchronize()
    kernel_ms.clear()
    launches[0] = 0
    ctx.stats_reset()

    c2_calls, c1_calls = step_calls()
    step_ms, e2e_s = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps
            rig.hist.zero_()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ms = rig.timed(one_step)
            h = rig.hist.cpu()                 # the step's result back on the host
            st = ctx.status()
            e2e_s.append(time.perf_counter() - t0)
            step_ms.append(ms)
            if any(st):
                raise RuntimeError(f"device status {st}")
    stats = ctx.stats()
    clocks = clk.summary()

    # the step's result, checked by what holds at any size: both forms agree
    # and every byte of the file is counted once (bit-exact parity with the
    # oracle is the GPU tests' job; the CPU-baseline leg below also compares
    # this histogram with the oracle's when it runs)
    c1_hist = h[0].numpy().view(np.uint32)
    if not (np.array_equal(c1_hist, h[1].numpy().view(np.uint32)) and int(c1_hist.sum(dtype=np.uint64)) == C1_BYTES):
        raise RuntimeError("C1 histograms of the plain and batched forms differ or miss bytes")
    # the C1 configuration (4 MiB, 64 work-groups x 256 threads, 4 KiB preads)
    # in its plain and batched forms, from the kernels of the timed steps
    c1_forms = {}
    for kname, form in (("c1_plain_kernel", "plain"), ("c1_batched_kernel", "batched")):
        ms_list = kernel_ms.get(kname, [])
        if ms_list:
            k_ms = statistics.median(ms_list)
            c1_forms[form] = {"kernel_ms": round(k_ms, 3), "GB_per_s": round(C1_BYTES / (k_ms * 1e-3) / 1e9, 2),
                              "preads_per_s": round(C1_BYTES // C1_CHUNK / (k_ms * 1e-3), 1),
                              "histogram_checked": "forms agree, every byte counted"}

    tot_ms, e2e_tot = reduce_max([sum(step_ms), sum(e2e_s)], dev)
    calls_step = c2_calls + c1_calls
    value = job_value(world, calls_step * args.steps, tot_ms * 1e-3)

    # ---- profile pass (untimed): per-combination rate and latency at 2^20,
    # latency of the plain form at every size, plain vs batched forms,
    # pread+scan GB/s at 1 GiB and over the C3 corpus
    # Each combination runs PROFILE_REPEATS times: rate and latency are the
    # median run's, `ms_best` the fastest (host cores are shared, and one
    # run can land on a slow stretch); the work-item phases are the best run's,
    # like the host-only probe it is compared with (best of 3).
    sweep = {}
    n = max(SIZES)
    plain_phases = None
    for name, g, bt, relaxed, nb in COMBOS:
        is_plain = combo_key(name, relaxed, nb) == combo_key("work-item", False, False)
        runs = []
        for _ in range(PROFILE_REPEATS):
            ctx.latency(clear=True)
            st0 = ctx.stats() if is_plain else None
            ms = rig.timed(lambda: rig.c2(n, g, bt, relaxed, nb))
            runs.append((ms, ctx.latency(clear=True), service_phases(st0, ctx.stats()) if is_plain else None))
        runs.sort(key=lambda t: t[0])
        ms, lat, _ = runs[len(runs) // 2]
        if is_plain:
            plain_phases = runs[0][2]
        calls = calls_for(g, bt, n)
        sweep[combo_key(name, relaxed, nb)] = {
            "ms": round(ms, 3), "ms_best": round(runs[0][0], 3), "syscalls_per_s": round(calls / (ms * 1e-3), 1),
            "requests_per_s": round(n / (ms * 1e-3), 1),
            "p50_us": round(pctl(lat, 50) / 1e3, 2) if len(lat) else None,
            "p99_us": round(pctl(lat, 99) / 1e3, 2) if len(lat) else None}
    # per-call latency of the C1 forms (the median of PROFILE_REPEATS runs):
    # for the batched form a call lasts from its issue to the wait that
    # collects it, so reads kept in flight while a chunk is scanned count
    for form, fv in (("plain", G.FORM_PLAIN), ("batched", G.FORM_BATCHED)):
        if form not in c1_forms:
            continue
        runs = []
        for _ in range(PROFILE_REPEATS):
            ctx.latency(clear=True)
            ms = rig.timed(lambda: rig.c1(fv))
            runs.append((ms, ctx.latency(clear=True)))
        runs.sort(key=lambda t: t[0])
        lat = runs[len(runs) // 2][1]
        c1_forms[form].update({"p50_us": round(pctl(lat, 50) / 1e3, 2) if len(lat) else None,
                               "p99_us": round(pctl(lat, 99) / 1e3, 2) if len(lat) else None})
    lat_by_size = {}
    for nn in SIZES:
        ctx.latency(clear=True)
        rig.c2(nn, 0, 256, False, False)
        lat = ctx.latency(clear=True)
        lat_by_size[str(nn)] = {"p50_us": round(pctl(lat, 50) / 1e3, 2), "p99_us": round(pctl(lat, 99) / 1e3, 2)}
    plain = sweep[combo_key("work-item", False, False)]
    batched_key = max((k for k in sweep if "relaxed" in k), key=lambda k: sweep[k]["requests_per_s"])
    batched = sweep[batched_key]
    # the same 2^20 work-item pwrites served call by call (Sec. 4.2 without
    # coalescing: no merging, batches of one doorbell entry) beside the
    # batched and merged service of the timed step
    per_call = per_call_service(G, rig, local, step_cfg["service_threads"], n)

    # The work-item kernels are bound by the service threads' rate, not by the
    # link: their calls/s against the ceiling of the same requests published
    # by a host thread (no GPU in the loop; same threads and batch size).
    torch.cuda.synchronize()
    n_probe = SIZES[-1]
    probes_run = []
    for _ in range(3):
        st0 = ctx.stats()
        rate = ctx.service_probe(rig.fds[n_probe], rig.c2_stage, 64, n_probe)
        probes_run.append((rate, service_phases(st0, ctx.stats())))
    ceiling, probe_phases = max(probes_run, key=lambda t: t[0])
    # best of the GPU path's runs against the probe's best; the median beside it
    plain_best = round(n / (plain["ms_best"] * 1e-3), 1)
    service_roofline = {"bound": "host_service", "kernel": "c2_pwrite_kernel<work-item,strong,blocking>",
                        "threads": n_probe, "achieved": plain_best, "achieved_median": plain["syscalls_per_s"],
                        "peak": round(ceiling, 1), "unit": "calls/s", "frac": round(plain_best / ceiling, 4),
                        "frac_median": round(plain["syscalls_per_s"] / ceiling, 4),
                        "achieved_source": f"best of {PROFILE_REPEATS} runs of the 2^20-thread kernel",
                        "peak_source": "genesys_service_probe: the same 2^20 64-byte pwrites published by a host "
                                       "thread, same service threads and batch size, best of 3 (measured)",
                        # where each request's service time goes, GPU in the loop against the probe
                        "service_ns_per_request": {"gpu_path": plain_phases, "host_probe": probe_phases}}
    # The probe above rings its doorbells in file order, so a batch is one
    # merged call; GPU warps ring theirs interleaved and their batches merge
    # about a warp per call.  The same calls in that order, for context (the
    # frac above stays against the file-order ceiling).
    try:
        runs = []
        for _ in range(2):
            st0 = ctx.stats()
            r_il = ctx.service_probe(rig.fds[n_probe], rig.c2_stage, 64, n_probe, run=32, stride=8)
            runs.append((r_il, service_phases(st0, ctx.stats())))
        il_peak, il_phases = max(runs, key=lambda t: t[0])
        service_roofline["warp_interleaved_order"] = {
            "peak": round(il_peak, 1), "frac": round(plain_best / il_peak, 4),
            "frac_median": round(plain["syscalls_per_s"] / il_peak, 4),
            "order": "doorbells in runs of 32 calls (a warp), neighbouring runs 1/8 of a round apart (the 8 warps "
                     "of a 256-thread block), best of 2 (measured)",
            "service_ns_per_request": il_phases}
    except Exception as e:  # reported in the line, never hidden
        service_roofline["warp_interleaved_order"] = {"error": f"{type(e).__name__}: {e}"}
    # Coarse-grain pwrites move 64 bytes per thread through one merged Linux
    # call per group: their bound is the host's write bandwidth into the file
    # (one tmpfs inode, writers serialised), measured here with the same
    # buffer and file by one host thread.
    host_write, host_chunk = host_pwrite_peak(rig.fds[n_probe], rig.c2_stage, n_probe * 64)
    coarse = sweep[combo_key("wg1024", True, False)]
    coarse_gbs = n_probe * 64 / (coarse["ms_best"] * 1e-3) / 1e9
    coarse_median = n_probe * 64 / (coarse["ms"] * 1e-3) / 1e9
    coarse_roofline = {"bound": "host_file_write", "kernel": "c2_pwrite_kernel<work-group,relaxed,blocking>",
                       "threads": n_probe, "group": 1024, "achieved": round(coarse_gbs, 3),
                       "achieved_median": round(coarse_median, 3), "peak": round(host_write, 3), "unit": "GB/s",
                       "frac": round(coarse_gbs / host_write, 4), "frac_median": round(coarse_median / host_write, 4),
                       "achieved_source": f"best of {PROFILE_REPEATS} runs",
                       "peak_source": f"one host thread writing the same 64 MiB from the same pinned buffer to the "
                                      f"same tmpfs file with pwrite calls of 256 KiB-64 MiB, best of 3 each (best: "
                                      f"{host_chunk >> 10} KiB calls; measured)"}
    link = host_link_peak(torch, sm=True)
    link["round_trip_ns"] = G.link_pingpong(local, rounds=20000)  # GPU <-> host flag, the floor of a blocking call
    probes = host_probes(torch, local, rig.scan_path)
    checks = {"c2_files": [(nn, os.path.join(rig.d, f"c2_{nn}.bin")) for nn in SIZES]}
    extras = profile_extras(args, rig, local, rank, link, checks) if args.extras else {}
    # dominant kernel of the timed region and its host-link roofline
    tot = {k: sum(v) for k, v in kernel_ms.items()}
    dom = max(tot, key=tot.get)
    avg_ms = statistics.mean(kernel_ms[dom])
    # algorithmic host-link bytes per launch of the dominant kernel, averaged
    # over the sizes it ran at (the method's own traffic: per GPU thread its
    # 64-byte payload; per call its 64-byte slot and its 8-byte result - 136 B
    # per work-item call; the doorbell entry is this design's, not counted)
    if dom.startswith("c2_pwrite_kernel"):
        gname = dom.split("<")[1].split(",")[0]
        gr = {v: k for k, v in G.GRAN_NAMES.items()}[gname]
        sel = [(nn, g, bt) for nn in SIZES for name, g, bt, relaxed, nb in COMBOS
               if g == gr and ("relaxed" if relaxed else "strong") in dom and ("nonblocking" in dom) == nb]
        alg_bytes = statistics.mean(nn * 64 + calls_for(g, bt, nn) * ALG_BYTES_PER_CALL for nn, g, bt in sel)
        units = statistics.mean(nn for nn, _, _ in sel)
    else:
        alg_bytes = C1_BYTES + (C1_BYTES // C1_CHUNK) * ALG_BYTES_PER_CALL
        units = C1_BYTES
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    # the kernel moves its bytes with its own SM stores (pwrite payloads and
    # slots) or loads (preads): the SMs' zero-copy rate over the link is its
    # ceiling; the copy engines' rate is reported beside it
    c2 = dom.startswith("c2")
    copy_peak = link["d2h"] if c2 else link["h2d"]
    peak = link.get("sm_write" if c2 else "sm_read") or copy_peak
    roofline = {"bound": "host_link", "kernel": dom, "achieved": round(achieved, 3), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 5), "traffic": load_traffic(dom, units),
                "peak_source": ("the SMs' zero-copy " + ("stores" if c2 else "loads") + " over 1 GiB of pinned memory "
                                "(genesys_link_stream) in this run (of measured)")
                if peak != copy_peak else "pinned cudaMemcpy sweep in this run, best at >= 64 MiB (of measured)",
                "peak_copy_engine": copy_peak, "frac_copy_engine": round(achieved / copy_peak, 5),
                "alg_bytes_per_launch": int(alg_bytes), "avg_launch_ms": round(avg_ms, 4),
                "share_of_timed_device_time": round(tot[dom] / sum(tot.values()), 4),
                "service": service_roofline, "coarse": coarse_roofline}

    cpu = cpu_baseline_sample(budget_s=20.0, c1_hist=c1_hist) if rank == 0 and args.extras else None
    if cpu is not None and cpu.get("c1_histogram_equals_oracle") is False:
        raise RuntimeError("the step's C1 histogram differs from the oracle's: no bench line")
    # the full-size C4 and C5 results against the oracle (after every GPU
    # measurement; rank 0)
    ochecks = oracle_checks(checks) if rank == 0 and args.extras else {"ran": False}

    line = {
        "metric": "GPU syscalls/s (C2 pwrite invocation sweep + C1 pread pass)",
        "value": round(value, 1), "unit": "syscalls/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 3),
        # the step's kernels alone (device time); the rest of ms_per_step is
        # launching, synchronising and draining between them
        "kernel_ms_per_step": round(sum(tot.values()) / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "threads": SIZES, "combinations": len(COMBOS), "kernels_per_step": len(SIZES) * len(COMBOS) + 2,
                   "syscalls_per_step": calls_step, "service_threads": step_cfg["service_threads"],
                   "coalesce_max": step_cfg["coalesce_max"], "poll_max_ns": step_cfg["poll_max_ns"],
                   "n_slots": step_cfg.get("n_slots", 0) or "2048 per SM",
                   "l2": "256 MiB device buffer written between timed steps (L2 flush)",
                   "parallelism": f"replicas x{world}"},
        "requests_per_s": round(job_value(world, (sum(SIZES) * len(COMBOS) + c1_calls) * args.steps, tot_ms * 1e-3), 1),
        "forms": {"plain_blocking_strong": {"combo": "work-item/strong/blocking", **plain},
                  "batched": {"combo": batched_key, **batched},
                  "plain_per_call_service": per_call},
        "plain_latency_by_threads": lat_by_size,
        "c1_4MiB": c1_forms,
        "sweep_2p20": sweep,
        **extras,
        "autotuned_step": {"best": step_cfg, "table": step_table},
        "host_link_GB_per_s": link,
        "probes": probes,
        "service": {k: stats[k] for k in ("requests", "os_calls", "batches", "bytes", "failed", "busy_ns",
                                          "pickup_ns", "order_ns", "complete_ns")},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(job_value(world, calls_step * args.steps, e2e_tot), 1), "unit": "syscalls/s",
                "h2d_bytes_per_step": 2 * C1_BYTES,
                "d2h_bytes_per_step": sum(SIZES) * 64 * len(COMBOS) + 2 * 1024 + 32},
        "clocks": clocks,
        "gpu_launches": launches[0],
        "oracle_checks": ochecks,
    }
    line["summary"] = summarize(line)  # last key: the driver keeps the line's tail
    rig.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- oracle
def oracle_checks(checks: dict) -> dict:
    """The CPU-baseline leg's comparisons of full-size results with the
    oracle: every C4 reply at every offered rate (by digest; a missing reply
    counts as a mismatch) against the oracle's replay in client sequence
    order, and every request and the output file of the full C5 trace against
    the oracle's replay of each request (shared among the host's cores)."""
    import filecmp
    import numpy as np
    import oracle
    out = {"ran": True}
    if "c2_files" in checks:
        # the files the sweep wrote (every combination writes the same bytes)
        # against the oracle's pwrites of the same threads
        same = {}
        for n, path in checks["c2_files"]:
            ref = path + ".oracle"
            oracle.c2_pwrite(ref, n, 1, SEED_C2)
            same[str(n)] = bool(filecmp.cmp(path, ref, shallow=False))
            os.unlink(ref)
        out["c2_files_equal"] = all(same.values())
        out["c2_files_by_threads"] = same
    if "scan" in checks:
        path, hist = checks["scan"]
        out["scan_1GiB_histogram_equal"] = bool(np.array_equal(hist, oracle.c1_histogram(path, SCAN_CHUNK)))
    if "c4" in checks:
        # every reply that came back, against the oracle's replay in client
        # sequence order of the requests that reached the server (all of them
        # unless datagrams were lost: then exactly the server's received log)
        tr, per_rate = checks["c4"]
        t = time.perf_counter()
        want = reply_digests(oracle.c4_replay(tr))
        by_rate, checked = {}, 0
        for rate, (d, seen) in per_rate.items():
            n = len(d)
            replied = d != 0  # a missing reply has digest 0, a real one never does
            if seen is None or seen.all():
                w, idx = want[:n], np.arange(n)
            else:
                idx = np.nonzero(seen)[0]
                w = reply_digests(oracle.c4_replay(tr, idx))
            cmp = replied[idx]
            bad = int(np.count_nonzero(d[idx][cmp] != w[cmp]))
            checked += int(cmp.sum())
            by_rate[rate] = {"mismatched": bad, "requests_lost": int(n - len(idx)),
                             "replies_lost": int(np.count_nonzero(~replied[idx]))}
        out["c4_by_rate"] = by_rate
        out["c4_replies_checked"] = checked
        out["c4_replies_equal"] = bool(per_rate) and all(v["mismatched"] == 0 for v in by_rate.values())
        out["c4_oracle_s"] = round(time.perf_counter() - t, 2)
    if "c5" in checks:
        tr, runs = checks["c5"]
        ref = os.path.join(os.path.dirname(next(iter(runs.values()))[1]), "out_full.oracle")
        if os.path.exists(ref):
            os.unlink(ref)
        t = time.perf_counter()
        want = oracle.c5_trace_parallel(tr, ref)
        m = np.arange(8)[None, :] < tr.n_ops[:, None]
        per = {}
        for name, (res, path) in runs.items():
            n_bad = int(np.count_nonzero(((np.asarray(res) != want) & m).any(axis=1)))
            per[name] = {"mismatched_requests": n_bad, "output_file_equal": bool(filecmp.cmp(path, ref, shallow=False))}
        out.update({"c5_requests_checked": len(tr), "c5_by_form": per,
                    "c5_full_equal": all(v["mismatched_requests"] == 0 and v["output_file_equal"] for v in per.values()),
                    "c5_oracle_s": round(time.perf_counter() - t, 2), "c5_oracle_processes": os.cpu_count()})
    return out


def oracle_step(d, budget_s=None):
    """One step of the workload by the CPU oracle: the same sweep of pwrites
    (grouped as each granularity issues them) and the C1 preads.  Returns
    (syscalls, seconds, complete)."""
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


def cpu_baseline_sample(budget_s=20.0, c1_hist=None):
    """The oracle timed on a bounded sample of one step; given the GPU arm's
    C1 histogram, also whether it equals the oracle's for the same file."""
    import numpy as np
    import workloads
    d = workloads.scratch_dir("bench_oracle")
    calls, sec, full = oracle_step(d, budget_s)
    out = {"value": round(calls / sec, 1), "unit": "syscalls/s", "cores": 1, "kind": "oracle",
           "sample": ("one full step" if full else f"first {calls} calls of one step") +
                     " (C2 sweep + C1 preads), sequential C oracle, 1 thread",
           "host_cpus": os.cpu_count()}
    if c1_hist is not None:
        import oracle
        want = oracle.c1_histogram(workloads.c1_file(os.path.join(d, "c1.bin"), C1_BYTES, seed=workloads.SEED_C1),
                                   C1_CHUNK)
        out["c1_histogram_equals_oracle"] = bool(np.array_equal(np.asarray(c1_hist), want))
    return out


WORKLOAD = ("C2 invocation microbenchmark sweep: 2^10..2^20 threads x {work-item, warp, work-group 64/256/1024, "
            "kernel} x {strong, relaxed} x {blocking, non-blocking}, 64-byte pwrite per thread to a tmpfs file at "
            "gid*64; then C1 (4 MiB file, 4 KiB preads, 64 work-groups x 256 threads, 256-bin histogram, plain and "
            "batched)")


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
            "config": {"workload": WORKLOAD, "issued_by": "the sequential CPU oracle (one host thread)",
                       "threads": SIZES, "combinations": len(COMBOS), "syscalls_per_step": sum(step_calls())},
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
    ap.add_argument("--service-threads", type=int, default=4)
    ap.add_argument("--autotune", type=int, default=1, help="autotune the step's context knobs (cached)")
    ap.add_argument("--extras", type=int, default=1, help="0: only the timed step (for launch lists)")
    ap.add_argument("--coalesce-max", type=int, default=64, help="--only: service batch size")
    ap.add_argument("--poll-max-ns", type=int, default=2048, help="--only: largest completion-poll back-off")
    ap.add_argument("--coalesce-window-ns", type=int, default=0,
                    help="--only: how long a service thread waits for more requests after a batch's first")
    ap.add_argument("--only", default=None, help="run one case: c2:<grain>/<order>/<block>:<threads>, "
                                                 "c1:<plain|batched>:<bytes>, c3:<plain|batched>[:<first n files>], c4, c5, fig10, f4")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_genesys(args)


if __name__ == "__main__":
    main()
