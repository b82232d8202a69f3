"""Python binding of the B300 GPU system-call runtime (libgenesys.so).

Argument marshalling only: every step of the path - the device-side
invocation protocol, the CPU service threads and the scan kernels - runs in
libgenesys.so (C++ and sm_103a CUDA).  PyTorch is used for device memory and
streams.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1705_06965_b300.build``); importing this package without it
raises, there is no fallback.

Paper: Vesely et al., "GPU System Calls" (GENESYS), arXiv 1705.06965.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# GENESYS_LIBRARY=checked selects the build with device-side index checks
LIB_PATH = os.path.join(_PKG, "libgenesys_checked.so" if os.environ.get("GENESYS_LIBRARY") == "checked"
                        else "libgenesys.so")

# x86-64 system call numbers (<asm/unistd_64.h>)
SYS_read, SYS_write, SYS_close, SYS_mmap, SYS_munmap = 0, 1, 3, 9, 11
SYS_pread64, SYS_pwrite64, SYS_getpid = 17, 18, 39
SYS_sendto, SYS_recvfrom, SYS_recvmmsg, SYS_sendmmsg = 44, 45, 299, 307
NR_NOP, NR_CHECK_VISIBLE = 0x7F00, 0x7F01

GRAN_ITEM, GRAN_WARP, GRAN_GROUP, GRAN_KERNEL = 0, 1, 2, 3
GRAN_NAMES = {GRAN_ITEM: "work-item", GRAN_WARP: "warp", GRAN_GROUP: "work-group", GRAN_KERNEL: "kernel"}
REQ_BLOCKING, REQ_RELAXED, REQ_TICKET = 0x1, 0x8, 0x10
INIT_HOST_ONLY, INIT_NO_THREADS, INIT_ANY_SYSCALL = 0x1, 0x2, 0x4
FORM_PLAIN, FORM_BATCHED, FORM_WARP, FORM_HBM = 0, 1, 2, 3
ST_FIRST_ERROR, ST_TIMEOUTS, ST_FAILED_CALLS, ST_BAD_ARGS, ST_WORDS = 0, 1, 2, 3, 8

EINVAL, ENOMEM, ETIMEDOUT, ENODEV, EDEVICE, ECUDA = -22, -12, -110, -19, -1001, -1000
SIZEOF_DEV = 7  # GENESYS_SIZEOF_DEV

# every entry point declared in include/genesys.h
EXPORTS = [
    "genesys_config_default", "genesys_init", "genesys_shutdown", "genesys_device_view", "genesys_launch",
    "genesys_service", "genesys_drain", "genesys_stats_get", "genesys_stats_reset", "genesys_status",
    "genesys_latency", "genesys_staging", "genesys_staging_reset", "genesys_last_error", "genesys_emulate_call",
    "genesys_c1_histogram", "genesys_c2_pwrite", "genesys_visibility_probe", "genesys_last_launch_ms",
    "genesys_c3_wordcount", "genesys_c3_wordcount_noalloc", "genesys_serve_config_default", "genesys_c5_serve",
    "genesys_reclaim", "genesys_mmap_reserve", "genesys_kv_start", "genesys_kv_stop", "genesys_kv_value",
    "genesys_kv_client", "genesys_c6_permute", "genesys_gpu_call", "genesys_echo_start", "genesys_echo_stop",
    "genesys_echo_client", "genesys_service_probe", "genesys_link_pingpong", "genesys_link_stream",
    "genesys_service_restart",
    "genesys_trace_read", "genesys_sizeof", "genesys_service_health", "genesys_service_probe_order",
    "genesys_stats", "genesys_graph_launches", "genesys_check_pread_cap", "genesys_kv_received",
]


class GenesysError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what} failed ({code}): {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("n_slots", ctypes.c_uint32), ("n_service_threads", ctypes.c_uint32),
        ("service_cpus", ctypes.POINTER(ctypes.c_int32)), ("staging_bytes", ctypes.c_uint64),
        ("coalesce_window_ns", ctypes.c_uint64), ("coalesce_max", ctypes.c_uint32), ("merge", ctypes.c_uint32),
        ("device_deadline_ns", ctypes.c_uint64), ("lat_samples", ctypes.c_uint32), ("flags", ctypes.c_uint32),
        ("idle_spin_ns", ctypes.c_uint64), ("poll_min_ns", ctypes.c_uint32), ("poll_max_ns", ctypes.c_uint32),
        ("trace_capacity", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
    ]


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("n_streams", ctypes.c_uint32),
                ("staging_budget", ctypes.c_uint64), ("hbm_budget", ctypes.c_uint64),
                ("slot_budget", ctypes.c_uint32), ("block_threads", ctypes.c_uint32), ("min_part", ctypes.c_uint32),
                ("use_graphs", ctypes.c_uint32), ("pread_to_hbm", ctypes.c_uint32),
                ("honor_arrivals", ctypes.c_uint32), ("reserve_mmaps", ctypes.c_uint32),
                ("timeout_ns", ctypes.c_uint64), ("persistent", ctypes.c_uint32),
                ("persistent_blocks", ctypes.c_uint32)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("requests", "syscalls", "makespan_ns", "max_inflight",
                                               "admission_wait_ns", "graph_launches")]


C5_OP_DTYPE = np.dtype([("kind", "<u4"), ("file", "<u4"), ("off", "<u8"), ("len", "<u8"), ("seed", "<u8"),
                        ("out_off", "<u8")])
C5_REQ_DTYPE = np.dtype([("arrival_ns", "<u8"), ("threads", "<u4"), ("n_ops", "<u4"), ("ops", C5_OP_DTYPE, (8,))])


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("requests", "os_calls", "failed", "nonblocking_failed", "bytes", "batches", "busy_ns")] + [
        ("by_op", ctypes.c_uint64 * 8), ("op_ns", ctypes.c_uint64 * 8), ("op_max_ns", ctypes.c_uint64 * 8),
        ("mmap_new", ctypes.c_uint64), ("mmap_reused", ctypes.c_uint64), ("service_cpu_ns", ctypes.c_uint64),
        ("protocol_errors", ctypes.c_uint64), ("pickup_ns", ctypes.c_uint64), ("order_ns", ctypes.c_uint64),
        ("complete_ns", ctypes.c_uint64), ("empty_polls", ctypes.c_uint64), ("hole_polls", ctypes.c_uint64)]

    OPS = ("pread", "pwrite", "sendto", "recvfrom", "mmap", "munmap", "internal", "other")

    def as_dict(self) -> dict:
        d = {n: int(getattr(self, n)) for n, _ in self._fields_ if n not in ("by_op", "op_ns", "op_max_ns")}
        d["by_op"] = {k: int(v) for k, v in zip(self.OPS, self.by_op)}
        d["op_ns"] = {k: int(v) for k, v in zip(self.OPS, self.op_ns)}
        d["op_max_ns"] = {k: int(v) for k, v in zip(self.OPS, self.op_max_ns)}
        return d


_lib = None


def lib() -> ctypes.CDLL:
    """Load libgenesys.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1705_06965_b300.build` "
                          "(the GPU path has no fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32, i64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
    sig = {
        "genesys_config_default": (ctypes.c_int, [ctypes.POINTER(Config)]),
        "genesys_init": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(vp)]),
        "genesys_shutdown": (ctypes.c_int, [vp]),
        "genesys_device_view": (ctypes.c_int, [vp, vp]),
        "genesys_launch": (ctypes.c_int, [vp, vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.c_size_t,
                                          ctypes.POINTER(vp), u32, vp]),
        "genesys_service": (ctypes.c_int, [vp, u64]),
        "genesys_drain": (ctypes.c_int, [vp, u64]),
        "genesys_stats_get": (ctypes.c_int, [vp, ctypes.POINTER(Stats)]),
        "genesys_stats": (ctypes.c_int, [vp, ctypes.POINTER(Stats)]),
        "genesys_graph_launches": (ctypes.c_int, [vp, ctypes.POINTER(u64)]),
        "genesys_check_pread_cap": (ctypes.c_int, [vp, u64]),
        "genesys_stats_reset": (ctypes.c_int, [vp]),
        "genesys_status": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.c_int]),
        "genesys_latency": (ctypes.c_int, [vp, ctypes.POINTER(u64), u32, ctypes.POINTER(u32), ctypes.c_int]),
        "genesys_staging": (vp, [vp, ctypes.c_size_t]),
        "genesys_staging_reset": (ctypes.c_int, [vp]),
        "genesys_last_error": (ctypes.c_char_p, []),
        "genesys_emulate_call": (ctypes.c_int, [vp, u32, ctypes.POINTER(u64), u32, ctypes.POINTER(i64)]),
        "genesys_c1_histogram": (ctypes.c_int, [vp, ctypes.c_int, u64, u64, u32, u32, u32, vp, u64, vp, vp]),
        "genesys_c2_pwrite": (ctypes.c_int, [vp, ctypes.c_int, u64, u32, u32, u32, u32, u64, vp, u64, vp]),
        "genesys_visibility_probe": (ctypes.c_int, [vp, u64, u32, u32, u32, u64, vp, vp, vp]),
        "genesys_last_launch_ms": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "genesys_c3_wordcount": (ctypes.c_int, [vp, vp, vp, u32, vp, vp, u32, u64, u32, u32, u32, vp, u64, vp, vp]),
        "genesys_c3_wordcount_noalloc": (ctypes.c_int, [vp, vp, vp, u32, vp, vp, u32, u64, u32, u32, u32, vp, u64,
                                                         vp, vp]),
        "genesys_serve_config_default": (ctypes.c_int, [ctypes.POINTER(ServeConfig)]),
        "genesys_reclaim": (ctypes.c_int, [vp]),
        "genesys_mmap_reserve": (ctypes.c_int, [vp, vp, u32]),
        "genesys_kv_start": (ctypes.c_int, [vp, vp, vp, vp, u32, u32, u32, u32, ctypes.c_uint16, u64,
                                            ctypes.POINTER(vp)]),
        "genesys_kv_stop": (ctypes.c_int, [vp, u64, ctypes.POINTER(u64)]),
        "genesys_kv_value": (ctypes.c_int, [vp, u32, vp]),
        "genesys_kv_received": (ctypes.c_int, [vp, vp, u64]),
        "genesys_c6_permute": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, u64, u32, u32, u32, vp, u64, vp]),
        "genesys_gpu_call": (ctypes.c_int, [vp, u32, ctypes.POINTER(u64), u32, u32, vp, vp]),
        "genesys_kv_client": (ctypes.c_int, [vp, vp, u64, vp, ctypes.c_uint16, u32, u64, vp, vp, vp, vp]),
        "genesys_c5_serve": (ctypes.c_int, [vp, vp, u32, vp, u32, ctypes.c_int32, ctypes.POINTER(ServeConfig), vp, vp,
                                            ctypes.POINTER(ServeStats)]),
        "genesys_service_restart": (ctypes.c_int, [vp, u32, u64]),
        "genesys_sizeof": (u32, [ctypes.c_int]),
        "genesys_service_health": (ctypes.c_int, [vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "genesys_trace_read": (ctypes.c_int, [vp, vp, u32, ctypes.POINTER(u32), vp, u32, ctypes.POINTER(u32),
                                              ctypes.POINTER(i64)]),
        "genesys_link_pingpong": (ctypes.c_int, [ctypes.c_int, u32, u64, ctypes.POINTER(u64)]),
        "genesys_link_stream": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, u64, ctypes.c_int, u32, u32, u32,
                                               ctypes.POINTER(ctypes.c_double)]),
        "genesys_service_probe": (ctypes.c_int, [vp, ctypes.c_int, vp, u32, u64, ctypes.POINTER(u64)]),
        "genesys_service_probe_order": (ctypes.c_int, [vp, ctypes.c_int, vp, u32, u64, u32, u32,
                                                       ctypes.POINTER(u64)]),
        "genesys_echo_start": (ctypes.c_int, [vp, u32, u32, u32, u32, u32, ctypes.c_uint16, u64, ctypes.POINTER(vp)]),
        "genesys_echo_stop": (ctypes.c_int, [vp, u64, vp]),
        "genesys_echo_client": (ctypes.c_int, [ctypes.c_uint16, u32, u32, u64, u32, u32, u64, u64, u32, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _check_layouts(L)
    _lib = L
    return L


def _check_layouts(L) -> None:
    """Refuse a library built from another version of the headers: every
    structure this binding mirrors must have the library's size."""
    mine = {0: ctypes.sizeof(Config), 1: ctypes.sizeof(Stats), 2: ctypes.sizeof(ServeConfig),
            3: ctypes.sizeof(ServeStats), 4: TRACE_DEV_DTYPE.itemsize, 5: TRACE_HOST_DTYPE.itemsize,
            6: C5_REQ_DTYPE.itemsize}
    bad = {k: (v, int(L.genesys_sizeof(k))) for k, v in mine.items() if int(L.genesys_sizeof(k)) != v}
    if bad:
        raise ImportError(f"{LIB_PATH} was built from other headers than this binding (struct sizes "
                          f"binding/library: {bad}); rebuild it with `python -m paper_1705_06965_b300.build --force`")


def last_error() -> str:
    m = lib().genesys_last_error()
    return m.decode(errors="replace") if m else ""


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise GenesysError(rc, what, last_error())
    return rc


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


class Context:
    """A GENESYS context: syscall area, doorbell rings, staging arena and CPU
    service threads (genesys_init / genesys_shutdown)."""

    def __init__(self, device: int = 0, n_slots: int = 0, service_threads: int = 4,
                 staging_bytes: int = 256 << 20, coalesce_window_ns: int = 0, coalesce_max: int = 64,
                 merge: bool = True, deadline_ns: int = 2_000_000_000, lat_samples: int = 1 << 20,
                 host_only: bool = False, no_threads: bool = False, any_syscall: bool = False,
                 idle_spin_ns: int = 200_000_000, service_cpus=None, poll_min_ns: int = 256,
                 poll_max_ns: int = 2048, trace: int = 0):
        L = lib()
        cfg = Config()
        _check(L.genesys_config_default(ctypes.byref(cfg)), "genesys_config_default")
        cfg.n_slots = n_slots
        cfg.n_service_threads = service_threads
        self._cpus = None
        if service_cpus is not None:
            self._cpus = (ctypes.c_int32 * len(service_cpus))(*service_cpus)
            cfg.service_cpus = ctypes.cast(self._cpus, ctypes.POINTER(ctypes.c_int32))
        cfg.staging_bytes = staging_bytes
        cfg.coalesce_window_ns = coalesce_window_ns
        cfg.coalesce_max = coalesce_max
        cfg.merge = 1 if merge else 0
        cfg.device_deadline_ns = int(deadline_ns)
        cfg.lat_samples = lat_samples
        cfg.idle_spin_ns = int(idle_spin_ns)
        cfg.poll_min_ns = int(poll_min_ns)
        cfg.poll_max_ns = int(poll_max_ns)
        cfg.trace_capacity = int(trace)
        cfg.flags = (INIT_HOST_ONLY if host_only else 0) | (INIT_NO_THREADS if no_threads else 0) | (
            INIT_ANY_SYSCALL if any_syscall else 0)
        self.config = cfg
        self.host_only = host_only
        self.device = device
        h = ctypes.c_void_p()
        _check(L.genesys_init(ctypes.byref(cfg), device, ctypes.byref(h)), "genesys_init")
        self._h = h

    # -- lifetime
    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("context is shut down")
        return self._h

    def close(self) -> None:
        """Shut the context down.  Refused (GenesysError, the context stays
        open) while a KVServer or EchoServer started on it still runs."""
        if getattr(self, "_h", None):
            rc = lib().genesys_shutdown(self._h)
            if rc == EINVAL:  # refused: nothing was freed
                raise GenesysError(rc, "genesys_shutdown", last_error())
            self._h = None
            _check(rc, "genesys_shutdown")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_view(self) -> ctypes.Array:
        """The context's device view (genesys_device_view) as raw bytes, for
        kernels of one's own: pass it by value, or bind it for the
        handle-less genesys_syscall (genesys_syscall_bind)."""
        buf = ctypes.create_string_buffer(int(lib().genesys_sizeof(SIZEOF_DEV)))
        _check(lib().genesys_device_view(self.handle, buf), "genesys_device_view")
        return buf

    # -- staging arena (pinned, host-mapped: one address valid on both sides)
    def staging(self, nbytes: int) -> int:
        """Address of nbytes of the context's pinned host-mapped staging arena
        (usable by the host and by GPU code until staging_reset or close)."""
        p = lib().genesys_staging(self.handle, nbytes)
        if not p:
            raise GenesysError(ENOMEM, "genesys_staging", last_error())
        return int(p)

    def staging_reset(self) -> None:
        _check(lib().genesys_staging_reset(self.handle), "genesys_staging_reset")

    @staticmethod
    def host_view(addr: int, nbytes: int, dtype=np.uint8) -> np.ndarray:
        """numpy view (host side) of staging memory at `addr`.  It does not
        keep the memory alive: it is valid only while its context is open
        (reading it after close() reads freed memory)."""
        buf = (ctypes.c_uint8 * nbytes).from_address(addr)
        return np.frombuffer(buf, dtype=dtype)

    # -- service side
    def drain(self, timeout_ns: int = 10_000_000_000) -> None:
        _check(lib().genesys_drain(self.handle, timeout_ns), "genesys_drain")

    def service(self, timeout_ns: int) -> int:
        return _check(lib().genesys_service(self.handle, timeout_ns), "genesys_service")

    def stats(self) -> dict:
        s = Stats()
        _check(lib().genesys_stats(self.handle, ctypes.byref(s)), "genesys_stats")
        return s.as_dict()

    def graph_launches(self) -> int:
        """Launches made through GENESYS_LAUNCH_GRAPH on this context."""
        n = ctypes.c_uint64()
        _check(lib().genesys_graph_launches(self.handle, ctypes.byref(n)), "genesys_graph_launches")
        return int(n.value)

    def pread_cap(self, cap_bytes: int) -> None:
        """Checked library only (GENESYS_LIBRARY=checked): every pread the
        service threads make asks for at most cap_bytes (0 = no cap), so GPU
        callers meet short reads mid-file (genesys_check_pread_cap)."""
        _check(lib().genesys_check_pread_cap(self.handle, int(cap_bytes)), "genesys_check_pread_cap")

    def reclaim(self) -> None:
        """Unpin and unmap regions GPU code released with munmap (call when no
        kernel using this context runs)."""
        _check(lib().genesys_reclaim(self.handle), "genesys_reclaim")

    def stats_reset(self) -> None:
        _check(lib().genesys_stats_reset(self.handle), "genesys_stats_reset")

    def trace_read(self, calibrate: bool = True):
        """Copy out and clear the per-call trace (genesys_trace_read): device
        records (TRACE_DEV_DTYPE), host records (TRACE_HOST_DTYPE), and the host
        minus device clock offset in ns (None without calibration)."""
        cap = int(self.config.trace_capacity)
        dev = np.zeros(max(cap, 1), TRACE_DEV_DTYPE)
        host = np.zeros(max(cap, 1), TRACE_HOST_DTYPE)
        nd, nh, off = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
        _check(lib().genesys_trace_read(self.handle, dev.ctypes.data, cap, ctypes.byref(nd), host.ctypes.data, cap,
                                        ctypes.byref(nh), ctypes.byref(off) if calibrate else None),
               "genesys_trace_read")
        return dev[:min(nd.value, cap)], host[:min(nh.value, cap)], (off.value if calibrate else None)

    def service_health(self, stall_ns: int = 100_000_000) -> tuple:
        """(rings stalled for stall_ns with requests waiting, requests pending)
        (genesys_service_health)."""
        mask, pend = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().genesys_service_health(self.handle, stall_ns, ctypes.byref(mask), ctypes.byref(pend)),
               "genesys_service_health")
        return [r for r in range(64) if mask.value >> r & 1], int(pend.value)

    def service_restart(self, ring: int, pause_ns: int = 0) -> None:
        """Stop the service thread of `ring`, leave the ring unserved for
        pause_ns, start a new one (genesys_service_restart)."""
        _check(lib().genesys_service_restart(self.handle, ring, pause_ns), "genesys_service_restart")

    def service_probe(self, fd: int, payload: int, bytes_per_call: int, n_calls: int, run: int = 1,
                      stride: int = 1) -> float:
        """Service-thread ceiling for work-item pwrites (genesys_service_probe):
        the host publishes the requests itself; returns calls per second.
        run/stride > 1 ring the doorbells out of file order, as GPU warps do
        (genesys_service_probe_order)."""
        ns = ctypes.c_uint64()
        _check(lib().genesys_service_probe_order(self.handle, fd, payload, bytes_per_call, n_calls, run, stride,
                                                 ctypes.byref(ns)), "genesys_service_probe")
        return n_calls / (ns.value * 1e-9) if ns.value else float("inf")

    def status(self, clear: bool = True) -> list:
        out = (ctypes.c_int32 * ST_WORDS)()
        _check(lib().genesys_status(self.handle, out, 1 if clear else 0), "genesys_status")
        return list(out)

    def latency(self, clear: bool = True, cap: Optional[int] = None) -> np.ndarray:
        cap = self.config.lat_samples if cap is None else cap
        out = np.zeros(max(cap, 1), np.uint64)
        n = ctypes.c_uint32()
        _check(lib().genesys_latency(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                                     ctypes.byref(n), 1 if clear else 0), "genesys_latency")
        return out[:min(n.value, cap)]

    def last_launch_ms(self) -> float:
        """Device time of the last launched kernel (CUDA events around it)."""
        ms = ctypes.c_float()
        _check(lib().genesys_last_launch_ms(self.handle, ctypes.byref(ms)), "genesys_last_launch_ms")
        return float(ms.value)

    def emulate_call(self, nr: int, args=(), flags: int = REQ_BLOCKING) -> int:
        a = (ctypes.c_uint64 * 6)(*[int(x) & ((1 << 64) - 1) for x in list(args) + [0] * (6 - len(args))])
        r = ctypes.c_int64()
        _check(lib().genesys_emulate_call(self.handle, nr, a, flags, ctypes.byref(r)), "genesys_emulate_call")
        return r.value

    # -- workloads
    def c1_histogram(self, fd: int, file_bytes: int, hist_dev_ptr: int, staging: int, staging_bytes: int,
                     chunk: int = 4096, groups: int = 64, threads: int = 256, form: int = FORM_PLAIN,
                     stream=None) -> None:
        _check(lib().genesys_c1_histogram(self.handle, fd, file_bytes, chunk, groups, threads, form, staging,
                                          staging_bytes, hist_dev_ptr, _stream_handle(stream)),
               "genesys_c1_histogram")

    def c2_pwrite(self, fd: int, n_threads: int, gran: int, group_threads: int, relaxed: bool, nonblocking: bool,
                  seed: int, staging: int, staging_bytes: int, stream=None) -> None:
        _check(lib().genesys_c2_pwrite(self.handle, fd, n_threads, gran, group_threads, 1 if relaxed else 0,
                                       1 if nonblocking else 0, seed, staging, staging_bytes,
                                       _stream_handle(stream)), "genesys_c2_pwrite")

    def c3_wordcount(self, fds, file_bytes, queries, counts_dev_ptr: int, staging: int, staging_bytes: int,
                     chunk: int = 1 << 20, ctas: int = 296, threads: int = 512, form: int = FORM_BATCHED,
                     stream=None) -> None:
        """fds/file_bytes: sequences; queries: list of bytes (1..16 each)."""
        f = np.ascontiguousarray(np.asarray(fds, dtype=np.int32))
        sz = np.ascontiguousarray(np.asarray(file_bytes, dtype=np.uint64))
        q = np.zeros((max(len(queries), 1), 16), np.uint8)
        ql = np.zeros(max(len(queries), 1), np.uint8)
        for i, s in enumerate(queries):
            m = min(len(s), 16)                # longer queries are passed on for the library to reject
            q[i, :m] = np.frombuffer(s[:m], np.uint8)
            ql[i] = min(len(s), 255)
        _check(lib().genesys_c3_wordcount(self.handle, f.ctypes.data, sz.ctypes.data, len(f), q.ctypes.data,
                                          ql.ctypes.data, len(queries), chunk, ctas, threads, form, staging,
                                          staging_bytes, counts_dev_ptr, _stream_handle(stream)),
               "genesys_c3_wordcount")

    def c5_serve(self, arrival_ns, threads, n_ops, ops, in_fds, out_fd: int, **cfg):
        """Serve a trace (arrays of arrival ns, thread counts, op counts and a
        [n, 8] C5_OP_DTYPE op table).  cfg: ServeConfig fields.  Returns
        (results [n, 8] uint64, latency_ns [n] uint64, stats dict)."""
        n = len(threads)
        reqs = np.zeros(n, C5_REQ_DTYPE)
        reqs["arrival_ns"] = arrival_ns
        reqs["threads"] = threads
        reqs["n_ops"] = n_ops
        reqs["ops"] = np.asarray(ops).astype(C5_OP_DTYPE)
        sc = ServeConfig()
        _check(lib().genesys_serve_config_default(ctypes.byref(sc)), "genesys_serve_config_default")
        for k, v in cfg.items():
            setattr(sc, k, int(v))
        fds = np.ascontiguousarray(np.asarray(in_fds, dtype=np.int32))
        res = np.zeros((max(n, 1), 8), np.uint64)
        lat = np.zeros(max(n, 1), np.uint64)
        st = ServeStats()
        _check(lib().genesys_c5_serve(self.handle, reqs.ctypes.data, n, fds.ctypes.data, len(fds), out_fd,
                                      ctypes.byref(sc), res.ctypes.data, lat.ctypes.data, ctypes.byref(st)),
               "genesys_c5_serve")
        return res[:n], lat[:n], {f: int(getattr(st, f)) for f, _ in ServeStats._fields_}

    def gpu_call(self, nr: int, args=(), gran: int = GRAN_GROUP, threads: int = 128, stream=None) -> int:
        """Make one system call from GPU code; returns its result (>= 0 or -errno)."""
        import torch
        a = (ctypes.c_uint64 * 6)(*[int(x) & ((1 << 64) - 1) for x in list(args) + [0] * (6 - len(args))])
        out = torch.zeros(1, dtype=torch.int64, device=f"cuda:{self.device}")
        _check(lib().genesys_gpu_call(self.handle, nr, a, gran, threads, out.data_ptr(), _stream_handle(stream)),
               "genesys_gpu_call")
        return int(out.item())

    def c6_permute(self, fd: int, input_dev_ptr: int, perm_dev_ptr: int, n_blocks: int, iters: int, relaxed: bool,
                   nonblocking: bool, staging: int, staging_bytes: int, stream=None) -> None:
        _check(lib().genesys_c6_permute(self.handle, fd, input_dev_ptr, perm_dev_ptr, n_blocks, iters,
                                        1 if relaxed else 0, 1 if nonblocking else 0, staging, staging_bytes,
                                        _stream_handle(stream)), "genesys_c6_permute")

    def visibility_probe(self, n_threads: int, gran: int, group_threads: int, relaxed: bool, seed: int,
                         probe: int, violations_dev_ptr: int, stream=None) -> None:
        _check(lib().genesys_visibility_probe(self.handle, n_threads, gran, group_threads, 1 if relaxed else 0,
                                              seed, probe, violations_dev_ptr, _stream_handle(stream)),
               "genesys_visibility_probe")


KV_REPLY_STRIDE = 8 + 1024


class KVServer:
    """GPU key-value server (genesys_kv_start / genesys_kv_stop)."""

    def __init__(self, ctx: Context, keys, vlen0, vseed0, n_sockets: int = 16, batch: int = 64, threads: int = 256,
                 port_base: int = 47000, idle_timeout_ns: int = 20_000_000_000):
        self.keys = np.ascontiguousarray(np.asarray(keys, np.uint8))
        self.vlen0 = np.ascontiguousarray(np.asarray(vlen0, np.uint16))
        self.vseed0 = np.ascontiguousarray(np.asarray(vseed0, np.uint64))
        self.n_sockets, self.port_base = n_sockets, port_base
        self._ctx = ctx  # the server runs on the context: keep it alive
        h = ctypes.c_void_p()
        _check(lib().genesys_kv_start(ctx.handle, self.keys.ctypes.data, self.vlen0.ctypes.data,
                                      self.vseed0.ctypes.data, len(self.vlen0), n_sockets, batch, threads, port_base,
                                      idle_timeout_ns, ctypes.byref(h)), "genesys_kv_start")
        self._h = h

    def value(self, k: int) -> bytes:
        buf = ctypes.create_string_buffer(1024)
        n = _check(lib().genesys_kv_value(self._h, k, buf), "genesys_kv_value")
        return buf.raw[:n]

    def received(self, n: int) -> np.ndarray:
        """Which of the requests with seq 0 .. n-1 reached the server (bool
        array; genesys_kv_received): call after the load, before stop."""
        words = np.zeros(max((n + 31) // 32, 1), np.uint32)
        _check(lib().genesys_kv_received(self._h, words.ctypes.data, n), "genesys_kv_received")
        return np.unpackbits(words.view(np.uint8), bitorder="little")[:n].astype(bool)

    def stop(self, timeout_ns: int = 30_000_000_000) -> int:
        """Stop the server; returns the replies it sent.  On an error the
        server is kept (its kernel may still run) and stop can be called again."""
        served = ctypes.c_uint64()
        if self._h:
            _check(lib().genesys_kv_stop(self._h, timeout_ns, ctypes.byref(served)), "genesys_kv_stop")
            self._h = None
        return served.value

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


def kv_client(reqs: bytes, req_off, arrival_ns, port_base: int, n_sockets: int, timeout_ns: int = 20_000_000_000):
    """Run the UDP load generator; returns (replies list, latency_ns, stats dict)."""
    n = len(arrival_ns)
    off = np.ascontiguousarray(np.asarray(req_off, np.uint64))
    arr = np.ascontiguousarray(np.asarray(arrival_ns, np.uint64))
    # the library reads request j at reqs[req_off[j]:req_off[j + 1]], 24 bytes at least
    if len(off) != n + 1 or (n and (int(off[-1]) > len(reqs) or bool(np.any(np.diff(off) < 24)))):
        raise ValueError("req_off must hold n + 1 increasing offsets into reqs, 24 bytes or more apart")
    rb = ctypes.create_string_buffer(reqs, max(len(reqs), 1))
    out = np.zeros(max(n, 1) * KV_REPLY_STRIDE, np.uint8)
    rlen = np.zeros(max(n, 1), np.uint32)
    lat = np.zeros(max(n, 1), np.uint64)
    st = np.zeros(6, np.uint64)
    rc = lib().genesys_kv_client(rb, off.ctypes.data, n, arr.ctypes.data, port_base, n_sockets, timeout_ns,
                                 out.ctypes.data, rlen.ctypes.data, lat.ctypes.data, st.ctypes.data)
    names = ("received", "duplicates", "malformed", "send_errors", "max_send_late_ns", "span_ns")
    stats = {k: int(v) for k, v in zip(names, st)}
    stats["rc"] = rc
    reps = [out[j * KV_REPLY_STRIDE: j * KV_REPLY_STRIDE + int(rlen[j])].tobytes() for j in range(n)]
    return reps, lat[:n], stats


TRACE_DEV_DTYPE = np.dtype([("slot", "<u4"), ("seq", "<u4"), ("nr", "<u4"), ("gran", "<u4"), ("t_call", "<u8"),
                            ("t_publish", "<u8"), ("t_done", "<u8")])
TRACE_HOST_DTYPE = np.dtype([("slot", "<u4"), ("seq", "<u4"), ("t_pickup", "<u8"), ("t_done", "<u8")])


def latency_by_gran(dev) -> dict:
    """Per invocation granularity: blocking calls traced, and their call-to-
    result time p50/p99 (ns), from device trace records alone."""
    out = {}
    done = dev[dev["t_done"] > 0]
    for g, name in GRAN_NAMES.items():
        sel = done[done["gran"] == g]
        if len(sel):
            t = sel["t_done"].astype(np.int64) - sel["t_call"].astype(np.int64)
            out[name] = {"calls": int(len(sel)), "p50_ns": int(np.percentile(t, 50)),
                         "p99_ns": int(np.percentile(t, 99))}
    return out


def trace_breakdown(dev, host, host_minus_device_ns: int) -> dict:
    """Join device and host trace records by (slot, seq) and give the
    percentiles (ns) of each stage of a blocking call: claim (call to
    publish), queue (publish to CPU pickup), service (pickup to completion
    word), delivery (completion word to result seen), total (call to result)."""
    done = dev[dev["t_done"] > 0]
    key_h = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(host["slot"], host["seq"]))}
    rows = [(i, key_h[(int(a), int(b))]) for i, (a, b) in enumerate(zip(done["slot"], done["seq"]))
            if (int(a), int(b)) in key_h]
    if not rows:
        return {"joined": 0}
    di = np.array([r[0] for r in rows])
    hi = np.array([r[1] for r in rows])
    d, h = done[di], host[hi]
    off = np.int64(host_minus_device_ns)
    stages = {
        "claim": d["t_publish"].astype(np.int64) - d["t_call"].astype(np.int64),
        "queue": h["t_pickup"].astype(np.int64) - (d["t_publish"].astype(np.int64) + off),
        "service": h["t_done"].astype(np.int64) - h["t_pickup"].astype(np.int64),
        "delivery": (d["t_done"].astype(np.int64) + off) - h["t_done"].astype(np.int64),
        "total": d["t_done"].astype(np.int64) - d["t_call"].astype(np.int64),
    }
    out = {"joined": len(rows), "by_gran": latency_by_gran(dev)}
    known = d["t_publish"] > 0  # collected tickets do not record when they were published
    for k, v in stages.items():
        if k in ("claim", "queue"):
            v = v[known]
        if len(v):
            out[k] = {"p50_ns": int(np.percentile(v, 50)), "p99_ns": int(np.percentile(v, 99))}
    return out


ECHO_SINGLE, ECHO_BATCH = 0, 1
ECHO_PACKET_MAX, ECHO_MAX_BATCH, ECHO_STOP_BYTES = 65504, 64, 4


class EchoServer:
    """GPU UDP echo server (genesys_echo_start / genesys_echo_stop)."""

    def __init__(self, ctx: Context, n_sockets: int = 8, max_packet: int = ECHO_PACKET_MAX, form: int = ECHO_SINGLE,
                 batch: int = 16, threads: int = 256, port_base: int = 45000, idle_timeout_ns: int = 20_000_000_000):
        self.n_sockets, self.port_base = n_sockets, port_base
        self._ctx = ctx  # the server runs on the context: keep it alive
        h = ctypes.c_void_p()
        _check(lib().genesys_echo_start(ctx.handle, n_sockets, max_packet, form, batch, threads, port_base,
                                        idle_timeout_ns, ctypes.byref(h)), "genesys_echo_start")
        self._h = h

    def stop(self, timeout_ns: int = 30_000_000_000) -> dict:
        """Stop the server; returns its packet and byte counts.  On an error
        the server is kept (its kernel may still run) and stop can be called
        again."""
        st = np.zeros(2, np.uint64)
        if self._h:
            _check(lib().genesys_echo_stop(self._h, timeout_ns, st.ctypes.data), "genesys_echo_stop")
            self._h = None
        return {"packets": int(st[0]), "bytes": int(st[1])}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


def link_pingpong(device: int = 0, rounds: int = 2000, timeout_ns: int = 2_000_000_000) -> float:
    """Host-link flag round trip between a GPU thread and a host thread
    (genesys_link_pingpong); returns nanoseconds per round trip."""
    ns = ctypes.c_uint64()
    _check(lib().genesys_link_pingpong(device, rounds, timeout_ns, ctypes.byref(ns)), "genesys_link_pingpong")
    return float(ns.value)


def link_stream(host_ptr: int, nbytes: int, write=False, device: int = 0, blocks: int = 0,
                threads: int = 512, reps: int = 3) -> float:
    """Zero-copy host-link GB/s of the SMs reading (write False/0), writing
    (True/1) or both at once (2: half the blocks each way, the two directions'
    bytes summed) nbytes of pinned, host-mapped memory at host_ptr
    (genesys_link_stream); blocks 0 = 4 per SM."""
    import torch
    if blocks == 0:
        blocks = 4 * torch.cuda.get_device_properties(device).multi_processor_count
    gbs = ctypes.c_double()
    _check(lib().genesys_link_stream(device, host_ptr, nbytes, int(write), blocks, threads, reps,
                                     ctypes.byref(gbs)), "genesys_link_stream")
    return float(gbs.value)


def echo_client(port_base: int, n_sockets: int, packet_bytes: int, n_packets: int, window: int = 4,
                threads: int = 4, seed: int = 0x5EED0010, stall_ns: int = 0, send_stop: bool = True) -> dict:
    """Closed-loop UDP echo load generator (genesys_echo_client); returns its
    counters, and GB/s of echoed bytes over the first-send-to-last-reply span."""
    st = np.zeros(7, np.uint64)
    _check(lib().genesys_echo_client(port_base, n_sockets, packet_bytes, n_packets, window, threads, seed, stall_ns,
                                     int(send_stop), st.ctypes.data), "genesys_echo_client")
    names = ("sent", "echoed", "bad", "lost", "span_ns", "bytes", "send_errors")
    out = {k: int(v) for k, v in zip(names, st)}
    out["GB_per_s"] = out["bytes"] / out["span_ns"] if out["span_ns"] else None
    return out
