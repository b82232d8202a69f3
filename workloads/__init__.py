"""Seeded synthetic inputs for the GPU system-call workloads.

This module only makes inputs (files, query lists, request traces) and records
what it emitted.  It holds none of the method's arithmetic, and both the CUDA
path and the CPU oracle read what it writes.  Randomness is splitmix64
(Steele, Lea & Flood 2014) used counter-based, implemented in ``gen.c``.

Workloads (sizes of the full configurations; tests use scaled-down ones):

* C1 - one file of 4 MiB of splitmix64 stream bytes (seed 0x5EED0001), read with
  pread in 4 KiB chunks (the paper's pread microbenchmark, Sec. 6 / Fig. 5).
* C2 - no input file: each thread writes 64 bytes of the seed-0x5EED0002 stream
  at offset gid*64 (the pwrite microbenchmark of Sec. 4.1 / Sec. 6).
* C3 - a corpus of lowercase words (Zipf(1.1) over a 50k vocabulary, lognormal
  file sizes) with 64 query words (wordcount, Sec. 7.1).
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgen.so")

SEED_C1 = 0x5EED0001
SEED_C2 = 0x5EED0002
SEED_C3 = 0x5EED0003
SEED_C4 = 0x5EED0004
SEED_C5 = 0x5EED0005

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so beside it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _SO, src, "-lm"])
    return _SO


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.gen_splitmix64_at.restype = ctypes.c_uint64
        _lib.gen_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib.gen_stream_bytes.restype = None
        _lib.gen_stream_bytes.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64]
        _lib.gen_stream_file.restype = ctypes.c_int
        _lib.gen_stream_file.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint64]
        _lib.gen_corpus.restype = ctypes.c_int
        _lib.gen_corpus.argtypes = [
            ctypes.c_char_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
            ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.gen_vocab_word.restype = ctypes.c_int
        _lib.gen_vocab_word.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_char_p]
    return _lib


def splitmix64_at(seed: int, i: int) -> int:
    """i-th (0-based) output of a splitmix64 generator started at state `seed`."""
    return int(_L().gen_splitmix64_at(seed & MASK64, i & MASK64))


def stream_bytes(seed: int, nbytes: int, byte0: int = 0) -> bytes:
    """Bytes [byte0, byte0+nbytes) of the little-endian stream of `seed`."""
    buf = ctypes.create_string_buffer(max(nbytes, 1))
    _L().gen_stream_bytes(seed & MASK64, byte0, buf, nbytes)
    return buf.raw[:nbytes]


def scratch_dir(name: str) -> str:
    """A directory on tmpfs (the paper's pread microbenchmark reads tmpfs files)."""
    base = os.environ.get("GENESYS_DATA_DIR", "/dev/shm" if os.path.isdir("/dev/shm") else "/tmp")
    d = os.path.join(base, f"genesys_{os.getuid()}_{name}")
    os.makedirs(d, exist_ok=True)
    return d


def c1_file(path: str | None = None, nbytes: int = 4 << 20, seed: int = SEED_C1) -> str:
    """The C1 input: `nbytes` of the splitmix64 stream of `seed`."""
    if path is None:
        path = os.path.join(scratch_dir("c1"), f"c1_{seed:x}_{nbytes}.bin")
    if not (os.path.exists(path) and os.path.getsize(path) == nbytes):
        rc = _L().gen_stream_file(path.encode(), seed & MASK64, nbytes)
        if rc:
            raise OSError(-rc, f"gen_stream_file({path})")
    return path


@dataclass
class Corpus:
    dir: str
    paths: list
    sizes: np.ndarray            # uint64 [n_files]
    queries: list                # list[bytes]
    truth: np.ndarray            # uint64 [n_files, n_queries]: emitted tokens equal to each query
    tokens: np.ndarray           # uint64 [n_files]
    params: dict = field(default_factory=dict)

    @property
    def total_bytes(self) -> int:
        return int(self.sizes.sum())

    def truth_total(self) -> np.ndarray:
        return self.truth.sum(axis=0, dtype=np.uint64)

    def queries_packed(self) -> tuple[np.ndarray, np.ndarray]:
        """Queries as a [nq, 16] uint8 array (NUL padded) and a [nq] length array."""
        q = np.zeros((len(self.queries), 16), np.uint8)
        ln = np.zeros(len(self.queries), np.uint8)
        for i, s in enumerate(self.queries):
            q[i, :len(s)] = np.frombuffer(s, np.uint8)
            ln[i] = len(s)
        return q, ln


C3_FULL = dict(n_files=2000, median_bytes=256 * 1024, sigma=2.0, cap_bytes=64 << 20,
               vocab_n=50000, zipf_s=1.1, n_present=60, n_absent=4, seed=SEED_C3)
C3_SMALL = dict(n_files=48, median_bytes=24 * 1024, sigma=1.0, cap_bytes=512 << 10,
                vocab_n=2000, zipf_s=1.1, n_present=60, n_absent=4, seed=SEED_C3)


def corpus(params: dict | None = None, name: str | None = None, n_threads: int | None = None) -> Corpus:
    """Generate (or reuse, keyed by the parameters) a word corpus on tmpfs."""
    p = dict(C3_FULL if params is None else params)
    key = "_".join(f"{k}{p[k]}" for k in sorted(p))
    tag = name or "c3_" + hashlib.sha1(key.encode()).hexdigest()[:12]
    d = scratch_dir(tag)
    man = os.path.join(d, "manifest.json")
    if os.path.exists(man):
        with open(man) as f:
            m = json.load(f)
        if m.get("params") == p and all(os.path.exists(x) for x in m["paths"]):
            return Corpus(d, m["paths"], np.array(m["sizes"], np.uint64),
                          [bytes.fromhex(q) for q in m["queries"]],
                          np.array(m["truth"], np.uint64).reshape(len(m["paths"]), -1),
                          np.array(m["tokens"], np.uint64), p)
    n, nq = p["n_files"], p["n_present"] + p["n_absent"]
    sizes = np.zeros(n, np.uint64)
    qbuf = np.zeros(nq * 16, np.uint8)
    qlen = np.zeros(nq, np.uint8)
    truth = np.zeros(n * nq, np.uint64)
    tokens = np.zeros(n, np.uint64)
    nt = n_threads or max(1, min(32, os.cpu_count() or 1))
    rc = _L().gen_corpus(d.encode(), n, float(p["median_bytes"]), float(p["sigma"]), int(p["cap_bytes"]),
                         int(p["vocab_n"]), float(p["zipf_s"]), int(p["n_present"]), int(p["n_absent"]),
                         int(p["seed"]) & MASK64, nt, sizes.ctypes.data, qbuf.ctypes.data, qlen.ctypes.data,
                         truth.ctypes.data, tokens.ctypes.data)
    if rc:
        raise OSError(-rc, "gen_corpus")
    paths = [os.path.join(d, f"f{i:05d}.txt") for i in range(n)]
    queries = [bytes(qbuf[16 * i:16 * i + int(qlen[i])]) for i in range(nq)]
    with open(man, "w") as f:
        json.dump({"params": p, "paths": paths, "sizes": sizes.tolist(), "queries": [q.hex() for q in queries],
                   "truth": truth.tolist(), "tokens": tokens.tolist()}, f)
    return Corpus(d, paths, sizes, queries, truth.reshape(n, nq), tokens, p)


def vocab_word(seed: int, vocab_n: int, idx: int) -> bytes:
    buf = ctypes.create_string_buffer(16)
    n = _L().gen_vocab_word(seed & MASK64, vocab_n, idx, buf)
    if n < 0:
        raise OSError(-n, "gen_vocab_word")
    return buf.raw[:n]


# ------------------------------------------------------------------------ C5
# Mixed serving trace: requests (GPU kernels) arrive as a Poisson process;
# each has a log-uniform thread count and a list of 1..8 operations drawn
# pread 50% / pwrite 25% / mmap-fill-munmap 25%.

C5_OP = np.dtype([("kind", "<u4"), ("file", "<u4"), ("off", "<u8"), ("len", "<u8"), ("seed", "<u8"),
                  ("out_off", "<u8")])
C5_MAX_OPS = 8
OP_PREAD, OP_PWRITE, OP_MMAP = 0, 1, 2

C5_FULL = dict(n_requests=10000, rate_per_s=20000.0, n_files=16, file_bytes=32 << 20, seed=SEED_C5)
C5_SMALL = dict(n_requests=200, rate_per_s=50000.0, n_files=4, file_bytes=4 << 20, seed=SEED_C5)


@dataclass
class Trace:
    arrival_ns: np.ndarray     # uint64 [n]
    threads: np.ndarray        # uint32 [n]
    n_ops: np.ndarray          # uint32 [n]
    ops: np.ndarray            # C5_OP [n, 8]
    in_paths: list
    out_bytes: int             # size of the output file (sum of pwrite lengths)
    params: dict = field(default_factory=dict)

    def __len__(self):
        return len(self.threads)

    def subset(self, idx) -> "Trace":
        idx = np.asarray(idx)
        return Trace(self.arrival_ns[idx], self.threads[idx], self.n_ops[idx], self.ops[idx], self.in_paths,
                     self.out_bytes, self.params)


def c5_trace(params: dict | None = None) -> Trace:
    """Generate the mixed trace (numpy, seeded) and its input files on tmpfs."""
    p = dict(C5_FULL if params is None else params)
    rng = np.random.default_rng(p["seed"])
    n = p["n_requests"]
    arrival = np.cumsum(rng.exponential(1.0 / p["rate_per_s"], n)) * 1e9
    threads = np.floor(np.exp(rng.uniform(np.log(64), np.log(65537), n))).astype(np.uint32)
    n_ops = rng.integers(1, C5_MAX_OPS + 1, n).astype(np.uint32)
    ops = np.zeros((n, C5_MAX_OPS), C5_OP)
    out_off = 0
    fb = p["file_bytes"]
    for r in range(n):
        for k in range(int(n_ops[r])):
            kind = int(rng.choice(3, p=[0.5, 0.25, 0.25]))
            op = ops[r, k]
            op["kind"] = kind
            op["seed"] = int(rng.integers(0, 1 << 62))
            if kind == OP_PREAD:
                ln = int(rng.integers(4096, 262145))
                op["file"] = int(rng.integers(0, p["n_files"]))
                op["len"] = ln
                op["off"] = int(rng.integers(0, fb - ln + 1))
            elif kind == OP_PWRITE:
                ln = int(rng.integers(4096, 262145))
                op["len"] = ln
                op["out_off"] = out_off
                out_off += ln
            else:
                ln = int(np.exp(rng.uniform(np.log(64 << 10), np.log((16 << 20) + 1))))
                op["len"] = max(4096, ln // 4096 * 4096)
    d = scratch_dir("c5_%x_%d_%d" % (p["seed"], p["n_files"], fb))
    paths = [c1_file(os.path.join(d, f"in{f:02d}.bin"), fb, seed=p["seed"] + 1 + f) for f in range(p["n_files"])]
    return Trace(arrival.astype(np.uint64), threads, n_ops, ops, paths, out_off, p)


# ------------------------------------------------------------------------ C4
# Key-value serving over UDP: 1M 16-byte keys preloaded with values of
# 64..1024 bytes; requests GET (90%) / SET (10%) with Zipf(0.99) key popularity
# and Poisson arrivals.  All byte strings derive from splitmix64 streams.

C4_FULL = dict(n_keys=1 << 20, n_requests=1 << 20, zipf_s=0.99, get_frac=0.9, rate_per_s=200_000.0,
               seed=SEED_C4)
C4_SMALL = dict(n_keys=1 << 14, n_requests=20_000, zipf_s=0.99, get_frac=0.9, rate_per_s=100_000.0, seed=SEED_C4)
KV_GET, KV_SET, KV_STOP = 0, 1, 2
KV_VMIN, KV_VMAX = 64, 1024


def _sm_vec(seed: int, idx: np.ndarray) -> np.ndarray:
    """splitmix64_at(seed, idx) for an index array (numpy uint64 arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


@dataclass
class KVTrace:
    keys: np.ndarray          # uint8 [n_keys, 16]
    vlen0: np.ndarray         # uint16 [n_keys]: preload value lengths
    vseed0: np.ndarray        # uint64 [n_keys]: preload value = stream_bytes(vseed0[i], vlen0[i])
    op: np.ndarray            # uint8 [n]
    key_idx: np.ndarray       # uint32 [n]
    vlen: np.ndarray          # uint16 [n] (SET)
    vseed: np.ndarray         # uint64 [n] (SET value = stream_bytes(vseed[j], vlen[j]))
    arrival_ns: np.ndarray    # uint64 [n]
    params: dict = field(default_factory=dict)

    def __len__(self):
        return len(self.op)

    def value0(self, i: int) -> bytes:
        return stream_bytes(int(self.vseed0[i]), int(self.vlen0[i]))

    def values0_table(self, width: int = 1024) -> np.ndarray:
        """All preload values as a [n_keys, width] byte table (row i = value0(i),
        zero padded), generated in blocks of keys."""
        nk = len(self.vlen0)
        out = np.zeros((nk, width), np.uint8)
        w = np.arange(width // 8, dtype=np.uint64)
        col = np.arange(width)
        for a in range(0, nk, 1 << 16):
            b = min(nk, a + (1 << 16))
            with np.errstate(over="ignore"):
                z = self.vseed0[a:b, None].astype(np.uint64) + (w[None, :] + np.uint64(1)) * np.uint64(GAMMA)
                z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
                z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
                z = z ^ (z >> np.uint64(31))
            rows = z.astype("<u8").view(np.uint8).reshape(b - a, width)
            out[a:b] = np.where(col[None, :] < self.vlen0[a:b, None], rows, 0)
        return out


def kv_trace(params: dict | None = None) -> KVTrace:
    p = dict(C4_FULL if params is None else params)
    s = p["seed"]
    nk, n = p["n_keys"], p["n_requests"]
    kw = _sm_vec(s ^ 0x1111, np.arange(2 * nk, dtype=np.uint64)).reshape(nk, 2)
    keys = kw.view(np.uint8).reshape(nk, 16).copy()
    if len(np.unique(keys.view([("a", "<u8"), ("b", "<u8")]))) != nk:
        raise RuntimeError("duplicate keys")
    vlen0 = (KV_VMIN + _sm_vec(s ^ 0x2222, np.arange(nk)) % np.uint64(KV_VMAX - KV_VMIN + 1)).astype(np.uint16)
    vseed0 = _sm_vec(s ^ 0x3333, np.arange(nk))
    rng = np.random.default_rng(s)
    ranks = np.arange(1, nk + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** -p["zipf_s"])
    cdf /= cdf[-1]
    key_idx = np.searchsorted(cdf, rng.random(n), side="right").astype(np.uint32)
    key_idx = np.minimum(key_idx, nk - 1)
    op = np.where(rng.random(n) < p["get_frac"], KV_GET, KV_SET).astype(np.uint8)
    vlen = np.where(op == KV_SET, rng.integers(KV_VMIN, KV_VMAX + 1, n), 0).astype(np.uint16)
    vseed = _sm_vec(s ^ 0x4444, np.arange(n))
    arrival = (np.cumsum(rng.exponential(1.0 / p["rate_per_s"], n)) * 1e9).astype(np.uint64)
    return KVTrace(keys, vlen0, vseed0, op, key_idx, vlen, vseed, arrival, p)


def kv_request_bytes(trace: KVTrace, idx=None) -> tuple[bytes, np.ndarray]:
    """Request datagrams of a KV trace (in the given order), back to back, and
    their offsets (n + 1).  Layout: op u8, pad u8, vlen u16, seq u32, key[16],
    value[vlen] (SET)."""
    idx = np.arange(len(trace)) if idx is None else np.asarray(idx)
    parts, offs, pos = [], [], 0
    for j in idx:
        op, kl = int(trace.op[j]), int(trace.vlen[j])
        d = bytes([op, 0]) + kl.to_bytes(2, "little") + int(j).to_bytes(4, "little")
        d += trace.keys[trace.key_idx[j]].tobytes()
        if op == KV_SET:
            d += stream_bytes(int(trace.vseed[j]), kl)
        offs.append(pos)
        parts.append(d)
        pos += len(d)
    return b"".join(parts), np.array(offs + [pos], np.uint64)



# ------------------------------------------------------------------------ C6
# Block permutation study (Fig. 6): random input blocks of 8 KiB and one
# seeded byte permutation of a block.

SEED_C6 = 0x5EED0006
C6_BLOCK = 8192


def c6_inputs(n_blocks: int, seed: int = SEED_C6) -> tuple[np.ndarray, np.ndarray]:
    """(input bytes [n_blocks * 8192] uint8, permutation [8192] uint16): the
    input is the splitmix64 stream of `seed`; the permutation sorts the
    stream of seed+1 (a uniformly random permutation)."""
    data = np.frombuffer(stream_bytes(seed, n_blocks * C6_BLOCK), np.uint8).copy()
    keys = _sm_vec(seed + 1, np.arange(C6_BLOCK))
    perm = np.argsort(keys, kind="stable").astype(np.uint16)
    return data, perm
