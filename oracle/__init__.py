"""CPU oracle for the GPU system-call workloads (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA path:
``oracle.c`` is a plain sequential C program that issues the same Linux calls
(pread, pwrite, ...) on the same seeded inputs and computes every result by its
plain definition in exact integer arithmetic.  Each function cites the passage
of Vesely et al., "GPU System Calls" (arXiv 1705.06965) that it follows.

Pins (tests/test_oracle.py): brute force on tiny inputs, the published
splitmix64 and FNV vectors, a hand-counted golden file, generator-recorded
ground truth, chunk-size invariance and closed forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc; OpenMP only for the
    files-to-cores wordcount baseline)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _SO, src])
    return _SO


_lib = None


def _L():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.oracle_splitmix64_at.restype = ctypes.c_uint64
        L.oracle_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_c1_histogram.restype = ctypes.c_int64
        L.oracle_c1_histogram.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_void_p]
        L.oracle_c2_pwrite.restype = ctypes.c_int64
        L.oracle_c2_pwrite.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_c3_wordcount.restype = ctypes.c_int64
        L.oracle_c3_wordcount.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_c3_wordcount_omp.restype = ctypes.c_int64
        L.oracle_c3_wordcount_omp.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
        L.oracle_c4_replay.restype = ctypes.c_int64
        L.oracle_c4_replay.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_kv_index.restype = ctypes.c_int64
        L.oracle_kv_index.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
        L.oracle_kv_serve.restype = ctypes.c_int64
        L.oracle_kv_serve.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                      ctypes.c_void_p]
        L.oracle_udp_echo.restype = ctypes.c_int64
        L.oracle_udp_echo.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                      ctypes.c_void_p]
        L.oracle_c6_permute.restype = ctypes.c_int64
        L.oracle_c6_permute.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32,
                                        ctypes.c_char_p]
        L.oracle_c5_checksum.restype = ctypes.c_uint64
        L.oracle_c5_checksum.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.oracle_c5_request.restype = ctypes.c_int64
        L.oracle_c5_request.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p]
        _lib = L
    return _lib


def _check(r: int, what: str) -> int:
    if r < 0:
        raise OSError(-r, f"oracle {what}: {os.strerror(-r)}")
    return r


def splitmix64_at(seed: int, i: int) -> int:
    """(i+1)-th output of splitmix64 started at state `seed` (Steele et al. 2014)."""
    return int(_L().oracle_splitmix64_at(seed & ((1 << 64) - 1), i))


def c1_histogram(path: str, chunk: int = 4096) -> np.ndarray:
    """C1 (Sec. 6, Fig. 5 pread microbenchmark): 256-bin uint32 histogram of the
    file's bytes, read with pread in `chunk`-byte pieces."""
    h = np.zeros(256, np.uint32)
    _check(_L().oracle_c1_histogram(path.encode(), chunk, h.ctypes.data), "c1_histogram")
    return h


def c2_pwrite(path: str, n_threads: int, group: int = 1, seed: int = 0x5EED0002) -> int:
    """C2 (Sec. 4.1 / Sec. 5 pwrite at a granularity): write thread gid's 64-byte
    splitmix64 pattern at offset gid*64, one pwrite per `group` work-items.
    Returns the number of pwrite calls issued."""
    return _check(_L().oracle_c2_pwrite(path.encode(), n_threads, group, seed), "c2_pwrite")


def _paths_array(paths):
    arr = (ctypes.c_char_p * len(paths))(*[p.encode() for p in paths])
    return arr


def _queries_array(queries):
    q = np.zeros((len(queries), 16), np.uint8)
    ln = np.zeros(len(queries), np.uint8)
    for i, s in enumerate(queries):
        if not 0 < len(s) <= 16:
            raise ValueError("queries must be 1..16 bytes")
        q[i, :len(s)] = np.frombuffer(s, np.uint8)
        ln[i] = len(s)
    return q, ln


def c3_wordcount(paths, queries, chunk: int = 1 << 20, per_file: bool = False, threads: int = 0):
    """C3 (Sec. 7.1 wordcount): whole-token occurrences of each query word over the
    files (tokens split on ' ' and '\\n').  threads > 0 runs the paper's OpenMP
    files-to-cores CPU version instead of the sequential one."""
    pa = _paths_array(paths)
    q, ln = _queries_array(queries)
    counts = np.zeros(len(queries), np.uint64)
    if threads > 0:
        if per_file:
            raise ValueError("per_file needs the sequential oracle")
        tot = _check(_L().oracle_c3_wordcount_omp(pa, len(paths), q.ctypes.data, ln.ctypes.data, len(queries),
                                                  chunk, counts.ctypes.data, threads), "c3_wordcount_omp")
        return counts, tot
    pf = np.zeros((len(paths), len(queries)), np.uint64) if per_file else None
    tot = _check(_L().oracle_c3_wordcount(pa, len(paths), q.ctypes.data, ln.ctypes.data, len(queries), chunk,
                                          counts.ctypes.data, pf.ctypes.data if per_file else None),
                 "c3_wordcount")
    return (counts, tot, pf) if per_file else (counts, tot)


def c5_checksum(data: bytes) -> int:
    """C5 checksum: sum mod 2^64 of splitmix64's output function applied to
    w_i + (i+1)*gamma over the little-endian 64-bit words w_i (zero padded)."""
    buf = ctypes.create_string_buffer(data, max(len(data), 1))
    return int(_L().oracle_c5_checksum(buf, len(data)))


def c5_request(ops, n_ops: int, in_fds, out_fd: int) -> np.ndarray:
    """C5 (Sec. 7 file and memory calls): run one request's operations in order
    (pread+checksum, pwrite of a seeded stream, mmap-fill-checksum-munmap);
    returns one uint64 result per operation."""
    ops = np.ascontiguousarray(ops)
    fds = np.ascontiguousarray(np.asarray(in_fds, dtype=np.int32))
    res = np.zeros(max(n_ops, 1), np.uint64)
    _check(_L().oracle_c5_request(ops.ctypes.data, n_ops, fds.ctypes.data, out_fd, res.ctypes.data), "c5_request")
    return res[:n_ops]


def c5_trace(trace, out_fd: int, in_fds=None) -> np.ndarray:
    """All requests of a trace in arrival order; results [n, 8] (unused ops 0)."""
    import os as _os
    own = in_fds is None
    if own:
        in_fds = [_os.open(p, _os.O_RDONLY) for p in trace.in_paths]
    try:
        out = np.zeros((len(trace), 8), np.uint64)
        for r in range(len(trace)):
            n = int(trace.n_ops[r])
            out[r, :n] = c5_request(trace.ops[r], n, in_fds, out_fd)
        return out
    finally:
        if own:
            for fd in in_fds:
                _os.close(fd)


def _c5_share(job):
    """One share of c5_trace_parallel, run in a child process: requests
    lo .. hi-1, each alone, in order."""
    ops, n_ops, in_paths, out_path, lo = job
    import os as _os
    in_fds = [_os.open(p, _os.O_RDONLY) for p in in_paths]
    ofd = _os.open(out_path, _os.O_RDWR)
    try:
        res = np.zeros((len(n_ops), 8), np.uint64)
        for i in range(len(n_ops)):
            n = int(n_ops[i])
            res[i, :n] = c5_request(ops[i], n, in_fds, ofd)
        return lo, res
    finally:
        for fd in in_fds + [ofd]:
            _os.close(fd)


def c5_trace_parallel(trace, out_path: str, procs: int = 0) -> np.ndarray:
    """c5_trace with its requests shared among `procs` processes (default:
    every host core), started with spawn so that a process that uses CUDA can
    call it.  Each request still runs alone, its operations in order, as in
    c5_trace; requests only read their input files and write disjoint ranges
    of the output file, so the results and the file are c5_trace's (pinned in
    tests/test_oracle.py).  Returns results [n, 8] (unused ops 0)."""
    import multiprocessing as mp
    import os as _os
    n = len(trace)
    procs = procs or (_os.cpu_count() or 1)
    _os.close(_os.open(out_path, _os.O_CREAT | _os.O_RDWR, 0o644))
    bounds = np.unique(np.linspace(0, n, 4 * procs + 1).astype(np.int64))  # more shares than processes: uneven requests
    jobs = [(trace.ops[a:b], trace.n_ops[a:b], list(trace.in_paths), out_path, int(a))
            for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    out = np.zeros((n, 8), np.uint64)
    with mp.get_context("spawn").Pool(min(procs, max(len(jobs), 1))) as pool:
        for lo, res in pool.imap_unordered(_c5_share, jobs):
            out[lo:lo + len(res)] = res
    return out


def c4_replay(trace, idx=None):
    """C4 (Sec. 7.3 UDP service): the sequential server's reply to each request
    of the trace (in the given order, default seq order), as a list of bytes."""
    import workloads
    nk = len(trace.keys)
    vals = trace.values0_table()
    vlens = trace.vlen0.astype(np.uint16).copy()
    reqs, _ = workloads.kv_request_bytes(trace, idx)
    n = len(trace) if idx is None else len(idx)
    out = np.zeros(n * (8 + 1024) + 8, np.uint8)
    off = np.zeros(n + 1, np.uint64)
    keys = np.ascontiguousarray(trace.keys)
    rb = ctypes.create_string_buffer(reqs, max(len(reqs), 1))
    _check(_L().oracle_c4_replay(keys.ctypes.data, nk, vals.ctypes.data, vlens.ctypes.data, rb, n,
                                 out.ctypes.data, off.ctypes.data), "c4_replay")
    return [out[int(off[i]):int(off[i + 1])].tobytes() for i in range(n)]


def _udp_sockets(port_base: int, n: int):
    import socket
    socks = []
    try:
        for w in range(n):
            so = socket.socket(socket.AF_INET, socket.SOCK_DGRAM)
            socks.append(so)
            for opt, force in ((socket.SO_RCVBUF, 33), (socket.SO_SNDBUF, 32)):  # *BUFFORCE when permitted
                try:
                    so.setsockopt(socket.SOL_SOCKET, force, 64 << 20)
                except OSError:
                    so.setsockopt(socket.SOL_SOCKET, opt, 64 << 20)
            so.bind(("127.0.0.1", port_base + w))
    except OSError:
        for so in socks:
            so.close()
        raise
    return socks


class UdpServer:
    """A plain CPU server (Sec. 7.3) on 127.0.0.1:port_base + w, w < n_sockets,
    run by `threads` host threads (thread t answers sockets t, t + threads, ...)
    until every socket gets its stop datagram or idle_ns passes without one.
    kind "echo": each datagram goes back unchanged.  kind "kv": each request is
    applied like c4_replay to the table of `trace` (keys and preloaded values).
    The sockets are bound before the constructor returns."""

    def __init__(self, kind: str, port_base: int, n_sockets: int, threads: int = 1, trace=None,
                 max_packet: int = 65504, idle_ns: int = 10_000_000_000, values0=None):
        import threading
        self.socks = _udp_sockets(port_base, n_sockets)
        self.stats = np.zeros((threads, 2), np.uint64)
        L = _L()
        if kind == "kv":
            nk = len(trace.keys)
            self._keys = np.ascontiguousarray(trace.keys)
            self._order = np.zeros(max(nk, 1), np.uint32)
            L.oracle_kv_index(self._keys.ctypes.data, nk, self._order.ctypes.data)
            # values0: trace.values0_table() computed once by the caller (copied here)
            self.vals = trace.values0_table() if values0 is None else np.array(values0, np.uint8, copy=True)
            self.vlens = trace.vlen0.astype(np.uint16).copy()
            if threads != 1:
                raise ValueError("the key-value oracle server is single-threaded (one table, one order)")
        self._fds = [np.array([s.fileno() for s in self.socks[t::threads]], np.int32) for t in range(threads)]

        def run(t):
            fds = self._fds[t]
            st = self.stats[t]
            if kind == "echo":
                L.oracle_udp_echo(fds.ctypes.data, len(fds), max_packet, idle_ns, st.ctypes.data)
            else:
                L.oracle_kv_serve(fds.ctypes.data, len(fds), self._keys.ctypes.data, self._order.ctypes.data,
                                  len(self._keys), self.vals.ctypes.data, self.vlens.ctypes.data, idle_ns,
                                  st.ctypes.data)

        self._threads = [threading.Thread(target=run, args=(t,), daemon=True) for t in range(threads)]
        for th in self._threads:
            th.start()

    def join(self, timeout: float = 60.0) -> dict:
        for th in self._threads:
            th.join(timeout)
        for s in self.socks:
            s.close()
        return {"answered": int(self.stats[:, 0].sum()), "bytes": int(self.stats[:, 1].sum())}


def c6_permute(input_bytes: np.ndarray, perm: np.ndarray, iters: int, path: str) -> int:
    """C6 (Sec. 6, Fig. 6 block permutation): permute each 8 KiB block `iters`
    times (out[i] = in[perm[i]]) and pwrite it at its own offset; returns the
    number of pwrite calls."""
    a = np.ascontiguousarray(input_bytes, dtype=np.uint8)
    p = np.ascontiguousarray(perm, dtype=np.uint16)
    if a.size % 8192 or p.size != 8192:
        raise ValueError("input must be whole 8 KiB blocks, perm 8192 entries")
    return _check(_L().oracle_c6_permute(a.ctypes.data, a.size // 8192, p.ctypes.data, iters, path.encode()),
                  "c6_permute")
