"""Autotuner: picks the service-thread count, slot-area size, invocation
granularity and chunk size of a workload by measuring candidates on the
machine it runs on, and caches the winners.

The right values depend on the host as much as on the GPU: how many cores can
serve calls, how fast the host copies pread data, how many requests a batch
merges.  Each tuner runs every candidate through the library's own entry
points (CUDA-event timing, best of `repeats`), keeps a table of what it
measured and stores the winner in a JSON cache keyed by workload, GPU and host
core count (``GENESYS_AUTOTUNE_CACHE`` or ``~/.cache/genesys_b300/autotune.json``).
"""
from __future__ import annotations

import itertools
import json
import os
import time
from typing import Callable, Iterable

_DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "genesys_b300", "autotune.json")


def _machine_key() -> str:
    import torch
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|cpus{os.cpu_count()}"


class Autotuner:
    def __init__(self, cache_path: str | None = None):
        self.path = cache_path or os.environ.get("GENESYS_AUTOTUNE_CACHE", _DEFAULT_CACHE)
        try:
            with open(self.path) as f:
                self.cache = json.load(f)
        except (OSError, ValueError):
            self.cache = {}

    def key(self, workload: str, **shape) -> str:
        return workload + "|" + ",".join(f"{k}={shape[k]}" for k in sorted(shape)) + "|" + _machine_key()

    def lookup(self, key: str):
        hit = self.cache.get(key)
        return None if hit is None else hit["best"]

    def save(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1)
        os.replace(tmp, self.path)

    def tune(self, key: str, candidates: Iterable[dict], run: Callable[[dict], float], repeats: int = 2,
             force: bool = False):
        """Measure run(cfg) (seconds, lower is better) for every candidate;
        returns (best cfg, [(cfg, seconds)])."""
        if not force and key in self.cache:
            return self.cache[key]["best"], self.cache[key]["table"]
        table = []
        for cfg in candidates:
            try:
                t = min(run(cfg) for _ in range(repeats))
            except Exception as e:  # a candidate the machine cannot run is skipped
                table.append((cfg, None, str(e)[:200]))
                continue
            table.append((cfg, t))
        ok = [r for r in table if r[1] is not None]
        if not ok:
            raise RuntimeError(f"autotune {key}: no candidate ran")
        best = min(ok, key=lambda r: r[1])[0]
        self.cache[key] = {"best": best, "table": table, "when": time.time()}
        self.save()
        return best, table


def _fit_threads(candidates) -> tuple:
    """Service-thread counts that leave two host cores for the calling thread
    and the GPU driver (the smallest candidate is always kept)."""
    room = max(1, (os.cpu_count() or 1) - 2)
    fit = tuple(t for t in candidates if t <= room)
    return fit or (min(candidates),)


def grid(**axes) -> list[dict]:
    names = list(axes)
    return [dict(zip(names, vals)) for vals in itertools.product(*(axes[n] for n in names))]


def _timed(torch, fn) -> float:
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    fn()
    e.record()
    e.synchronize()
    return s.elapsed_time(e) * 1e-3


def tune_scan(device: int, fd: int, nbytes: int, tuner: Autotuner | None = None, force: bool = False,
              service_threads=(8, 12, 14), chunks=(128 << 10, 256 << 10, 512 << 10, 1 << 20),
              groups=(148, 296), forms=(0, 1, 2, 3), warp_chunks=(16 << 10, 64 << 10)):
    """pread + histogram scan: service threads x chunk x groups x form, where
    the form sets the invocation granularity (work-group plain or batched,
    or warp, which reads smaller chunks: `warp_chunks`) and where the chunk
    is counted (staging, or an HBM copy: form 3)."""
    import torch
    import paper_1705_06965_b300 as G
    tuner = tuner or Autotuner()
    service_threads = _fit_threads(service_threads)
    key = tuner.key("scan", nbytes=nbytes)
    hit = None if force else tuner.lookup(key)
    if hit:
        return hit
    hist = torch.zeros(256, dtype=torch.int32, device=f"cuda:{device}")
    table_all, best, best_t = [], None, None
    cands = [c for c in grid(chunk=chunks, groups=groups, form=[f for f in forms if f != 2])]
    if 2 in forms:
        cands += grid(chunk=warp_chunks, groups=groups, form=(2,))
    stage_bytes = max(c["groups"] * c["chunk"] * (32 if c["form"] == 2 else 2) for c in cands)
    for st in service_threads:
        with G.Context(device=device, service_threads=st, staging_bytes=stage_bytes + (1 << 20)) as ctx:
            stage = ctx.staging(stage_bytes)

            def run(cfg):
                fn = lambda: ctx.c1_histogram(fd, nbytes, hist.data_ptr(), stage, stage_bytes, chunk=cfg["chunk"],  # noqa
                                              groups=cfg["groups"], threads=1024, form=cfg["form"])
                fn()
                return _timed(torch, fn)

            for cfg in cands:
                t = min(run(cfg) for _ in range(2))
                c = dict(cfg, service_threads=st)
                table_all.append((c, t))
                if best_t is None or t < best_t:
                    best, best_t = c, t
    # the best setting of each form too, so that callers can compare forms
    by_form = {}
    for c, t in table_all:
        f = str(c["form"])
        if f not in by_form or t < by_form[f][1]:
            by_form[f] = (c, t)
    best = dict(best, by_form={f: c for f, (c, _) in by_form.items()})
    tuner.cache[key] = {"best": best, "table": table_all, "when": time.time()}
    tuner.save()
    return best


def tune_wordcount(device: int, fds, sizes, queries, tuner: Autotuner | None = None, force: bool = False,
                   service_threads=(8, 12, 14), chunks=(256 << 10, 1 << 20), ctas=(148, 296), forms=(0, 1)):
    """C3 wordcount: service threads x chunk x persistent blocks x form."""
    import numpy as np
    import torch
    import paper_1705_06965_b300 as G
    tuner = tuner or Autotuner()
    service_threads = _fit_threads(service_threads)
    total = int(np.asarray(sizes, np.uint64).sum())
    key = tuner.key("wordcount", files=len(sizes), bytes=total)
    hit = None if force else tuner.lookup(key)
    if hit:
        return hit
    counts = torch.zeros(len(queries), dtype=torch.int64, device=f"cuda:{device}")
    table_all, best, best_t = [], None, None
    stage_bytes = 2 * max(ctas) * (max(chunks) + 64)
    for st in service_threads:
        with G.Context(device=device, service_threads=st, staging_bytes=stage_bytes + (1 << 20)) as ctx:
            stage = ctx.staging(stage_bytes)
            for cfg in grid(chunk=chunks, ctas=ctas, form=forms):
                fn = lambda: ctx.c3_wordcount(fds, sizes, queries, counts.data_ptr(), stage, stage_bytes,  # noqa
                                              chunk=cfg["chunk"], ctas=cfg["ctas"], threads=512, form=cfg["form"])
                fn()
                t = min(_timed(torch, fn) for _ in range(2))
                c = dict(cfg, service_threads=st)
                table_all.append((c, t))
                if best_t is None or t < best_t:
                    best, best_t = c, t
    tuner.cache[key] = {"best": best, "table": table_all, "when": time.time()}
    tuner.save()
    return best


def tune_context(device: int, step: Callable, tuner: Autotuner | None = None, force: bool = False,
                 workload: str = "step", service_threads=(2, 4, 8), coalesce_max=(64, 256), n_slots=(0,),
                 staging_bytes: int = 256 << 20, setup: Callable | None = None):
    """Context-level knobs (service threads, batch size, slot-area size) for a
    callable step(ctx, state) that runs a workload through the context;
    setup(ctx) -> state allocates what the step needs."""
    import torch
    import paper_1705_06965_b300 as G
    tuner = tuner or Autotuner()
    key = tuner.key(workload)
    hit = None if force else tuner.lookup(key)
    if hit:
        return hit
    table_all, best, best_t = [], None, None
    for cfg in grid(service_threads=service_threads, coalesce_max=coalesce_max, n_slots=n_slots):
        with G.Context(device=device, service_threads=cfg["service_threads"], coalesce_max=cfg["coalesce_max"],
                       n_slots=cfg["n_slots"], staging_bytes=staging_bytes) as ctx:
            state = setup(ctx) if setup else None
            step(ctx, state)
            t = min(_timed(torch, lambda: step(ctx, state)) for _ in range(2))
        table_all.append((cfg, t))
        if best_t is None or t < best_t:
            best, best_t = cfg, t
    tuner.cache[key] = {"best": best, "table": table_all, "when": time.time()}
    tuner.save()
    return best


def tune_serve(device: int, ctx, trace, in_fds, out_fd: int, tuner: Autotuner | None = None, force: bool = False,
               min_parts=(4096, 16384, 65536), block_threads=(256, 1024), n_requests: int = 300,
               extra: dict | None = None):
    """C5 serving: the granularity of the request kernels' pread/pwrite calls
    (min_part: bytes per work-group call) x threads per block, measured as the
    makespan of the trace's first n_requests served back to back.  extra:
    serve settings every candidate shares (e.g. persistent=1 tunes the
    executor form on its own)."""
    import numpy as np
    tuner = tuner or Autotuner()
    extra = dict(extra or {})
    key = tuner.key("serve", requests=n_requests, min_parts=len(min_parts), block_threads=len(block_threads),
                    **{k: int(v) for k, v in sorted(extra.items())})
    hit = None if force else tuner.lookup(key)
    if hit:
        return hit
    sub = trace.subset(np.arange(min(n_requests, len(trace))))

    def run(cfg):
        _, _, st = ctx.c5_serve(sub.arrival_ns, sub.threads, sub.n_ops, sub.ops, in_fds, out_fd, honor_arrivals=0,
                                **cfg, **extra)
        return st["makespan_ns"] * 1e-9

    best, _ = tuner.tune(key, grid(min_part=min_parts, block_threads=block_threads), run, repeats=1, force=True)
    return best
