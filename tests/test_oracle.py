"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each pin is chosen so that a plausible mistake in the oracle - a dropped final
chunk or token, an off-by-one offset, a wrong byte order, a transposed
operand - fails at least one of them.
"""
import collections
import os
import re

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------------ splitmix64

def test_splitmix64_published_vector():
    # Published outputs of the splitmix64 reference implementation, state 0.
    for ln in _golden_lines("splitmix64_seed0.txt"):
        i, hx = ln.split()
        assert oracle.splitmix64_at(0, int(i)) == int(hx, 16)
        assert workloads.splitmix64_at(0, int(i)) == int(hx, 16)


# ------------------------------------------------------------------------- C1

def _write(path, data: bytes):
    with open(path, "wb") as f:
        f.write(data)
    return path


def test_c1_golden_abracadabra(tmp_path):
    lines = _golden_lines("c1_abracadabra.txt")
    content = lines[0].split(" ", 1)[1].encode()
    want = np.zeros(256, np.uint32)
    for ln in lines[1:]:
        b, c = ln.split()
        want[int(b)] = int(c)
    p = _write(tmp_path / "a.bin", content)
    for chunk in (1, 2, 3, 4096):
        assert np.array_equal(oracle.c1_histogram(str(p), chunk), want)


@pytest.mark.parametrize("size", [0, 1, 63, 64, 4095, 4096, 4097, 3 * 4096 + 17])
def test_c1_brute_force_and_chunk_invariance(tmp_path, size):
    rng = np.random.default_rng(size + 1)
    data = rng.integers(0, 256, size, dtype=np.uint8).tobytes()
    p = _write(tmp_path / "r.bin", data)
    brute = np.zeros(256, np.uint32)
    for b in data:                      # counting loop, one byte at a time
        brute[b] += 1
    for chunk in (1, 7, 4096, 1 << 20):
        h = oracle.c1_histogram(str(p), chunk)
        assert np.array_equal(h, brute), chunk
        assert int(h.sum()) == size


def test_c1_full_size_invariants():
    p = workloads.c1_file()
    h = oracle.c1_histogram(p, 4096)
    n = 4 << 20
    assert int(h.sum(dtype=np.uint64)) == n
    # splitmix64 bytes are close to uniform: every bin within 6 sigma of n/256
    mu, sd = n / 256, (n * (1 / 256) * (255 / 256)) ** 0.5
    assert np.all(np.abs(h.astype(np.float64) - mu) < 6 * sd)
    # the file's first 8 bytes are the first stream word, little-endian
    with open(p, "rb") as f:
        head = f.read(8)
    assert int.from_bytes(head, "little") == oracle.splitmix64_at(workloads.SEED_C1, 0)


def test_c1_missing_file_is_an_error(tmp_path):
    with pytest.raises(OSError):
        oracle.c1_histogram(str(tmp_path / "nope.bin"))


# ------------------------------------------------------------------------- C2

@pytest.mark.parametrize("n", [1, 31, 1024, 1000, 4096 + 5])
def test_c2_file_equals_stream_for_every_grouping(tmp_path, n):
    want = workloads.stream_bytes(workloads.SEED_C2, n * 64)
    for group in (1, 32, 64, 256, 1024, n):
        p = str(tmp_path / f"c2_{group}.bin")
        calls = oracle.c2_pwrite(p, n, group)
        assert calls == -(-n // group)
        with open(p, "rb") as f:
            got = f.read()
        assert len(got) == n * 64
        assert got == want, group


def test_c2_seed0_head_is_published_vector(tmp_path):
    p = str(tmp_path / "c2s0.bin")
    oracle.c2_pwrite(p, 1, 1, seed=0)
    with open(p, "rb") as f:
        head = f.read(24)
    words = [int.from_bytes(head[8 * k:8 * k + 8], "little") for k in range(3)]
    assert words == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ------------------------------------------------------------------------- C3

def _brute_wordcount(data: bytes, queries):
    toks = [t for t in re.split(rb"[ \n]", data) if t]
    c = collections.Counter(toks)
    return np.array([c[q] for q in queries], np.uint64)


def test_c3_golden_tiny(tmp_path):
    lines = _golden_lines("c3_tiny.txt")
    content = "\n".join(ln[len("content "):] for ln in lines if ln.startswith("content "))
    content = content.replace("\\n", "\n").encode()
    counts = [ln.split()[1:] for ln in lines if ln.startswith("count ")]
    queries = [q.encode() for q, _ in counts]
    want = np.array([int(c) for _, c in counts], np.uint64)
    p = _write(tmp_path / "t.txt", content)
    for chunk in (1, 2, 3, 5, 4096):
        got, tot = oracle.c3_wordcount([str(p)], queries, chunk=chunk)
        assert tot == len(content)
        assert np.array_equal(got, want), chunk


EDGE_FILES = [
    b"",
    b" ",
    b"\n\n  \n",
    b"cat",
    b"cat ",
    b" cat",
    b"cat\ncat cat\n\ncat",
    b"catcat cat cat1 ca t",
    b"abcdefghijklmnopqrstuvwxyz cat abcdefghijklmnop cat",   # tokens longer than 16
    b"abcdefghijklmnop",                                    # a 16-byte query token at EOF
]


def test_c3_edge_cases_brute_force(tmp_path):
    queries = [b"cat", b"ca", b"t", b"abcdefghijklmnop", b"dog"]
    for i, data in enumerate(EDGE_FILES):
        p = _write(tmp_path / f"e{i}.txt", data)
        want = _brute_wordcount(data, queries)
        for chunk in (1, 2, 3, 16, 4096):
            got, _ = oracle.c3_wordcount([str(p)], queries, chunk=chunk)
            assert np.array_equal(got, want), (data, chunk)


def test_c3_random_brute_force_multi_file(tmp_path):
    rng = np.random.default_rng(7)
    alphabet = np.frombuffer(b"ab \n", np.uint8)
    paths, datas = [], []
    for i in range(6):
        data = alphabet[rng.integers(0, 4, int(rng.integers(0, 3000)))].tobytes()
        paths.append(str(_write(tmp_path / f"m{i}.txt", data)))
        datas.append(data)
    queries = [b"a", b"b", b"ab", b"ba", b"aab", b"abab", b"bbbb"]
    want = sum(_brute_wordcount(d, queries) for d in datas)
    for chunk in (1, 5, 64, 1 << 20):
        got, tot = oracle.c3_wordcount(paths, queries, chunk=chunk)
        assert tot == sum(len(d) for d in datas)
        assert np.array_equal(got, want)
    omp, _ = oracle.c3_wordcount(paths, queries, chunk=64, threads=3)
    assert np.array_equal(omp, want)


def test_c3_matches_generator_ground_truth():
    # The generator records, as it writes each file, how many emitted tokens
    # equal each query; the oracle must find exactly those occurrences.
    c = workloads.corpus(workloads.C3_SMALL)
    got, tot, pf = c3 = oracle.c3_wordcount(c.paths, c.queries, chunk=4096, per_file=True)
    assert tot == c.total_bytes
    assert np.array_equal(pf, c.truth)
    assert np.array_equal(got, c.truth_total())
    # present words are found, absent words (the last four queries) only ever
    # as a truncated final token
    assert got[:60].sum() > 0
    # the query list holds distinct strings
    assert len(set(c.queries)) == len(c.queries)
    del c3


def test_c3_files_are_well_formed():
    c = workloads.corpus(workloads.C3_SMALL)
    for p, sz in zip(c.paths[:8], c.sizes[:8]):
        data = open(p, "rb").read()
        assert len(data) == int(sz)
        assert re.fullmatch(rb"[a-z \n]*", data)
        assert not data.startswith((b" ", b"\n"))
        assert b"  " not in data and b"\n\n" not in data and b" \n" not in data and b"\n " not in data


# ------------------------------------------------------------------------- C5

SM0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]   # published, state 0


def test_c5_checksum_zero_words_are_the_published_stream():
    # the checksum of k zero words is the sum of the first k outputs of
    # splitmix64 started at 0; a partial word is zero padded
    assert oracle.c5_checksum(b"\0" * 8) == SM0[0]
    assert oracle.c5_checksum(b"\0" * 16) == (SM0[0] + SM0[1]) % 2**64
    assert oracle.c5_checksum(b"\0" * 24) == sum(SM0) % 2**64
    assert oracle.c5_checksum(b"\0" * 20) == sum(SM0) % 2**64
    assert oracle.c5_checksum(b"") == 0


def test_c5_checksum_is_order_sensitive_and_word_local():
    a = bytes(range(64))
    b = bytearray(a)
    b[8:16], b[16:24] = a[16:24], a[8:16]           # swap two words: a different sum
    assert oracle.c5_checksum(a) != oracle.c5_checksum(bytes(b))
    c = bytearray(a)
    c[63] ^= 1                                       # one flipped bit changes it
    assert oracle.c5_checksum(a) != oracle.c5_checksum(bytes(c))


def _ops(*rows):
    ops = np.zeros(8, workloads.C5_OP)
    for k, r in enumerate(rows):
        for f, v in r.items():
            ops[k][f] = v
    return ops


def test_c5_ops_against_independent_paths(tmp_path):
    src = workloads.c1_file(str(tmp_path / "in.bin"), 100_000, seed=99)
    data = open(src, "rb").read()
    out = str(tmp_path / "out.bin")
    in_fd = os.open(src, os.O_RDONLY)
    out_fd = os.open(out, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
    try:
        ops = _ops({"kind": 0, "file": 0, "off": 1000, "len": 5000},
                   {"kind": 1, "len": 4099, "seed": 77, "out_off": 10},
                   {"kind": 2, "len": 65536, "seed": 5},
                   {"kind": 0, "file": 0, "off": 99_000, "len": 4096})      # short read at end of file
        res = oracle.c5_request(ops, 4, [in_fd], out_fd)
    finally:
        os.close(in_fd)
        os.close(out_fd)
    # pread: the checksum of the bytes a plain file read returns
    assert res[0] == oracle.c5_checksum(data[1000:6000])
    assert res[3] == oracle.c5_checksum(data[99_000:])
    # pwrite: the byte count, and the file holds the generator's stream at out_off
    assert res[1] == 4099
    got = open(out, "rb").read()
    assert got[10:] == workloads.stream_bytes(77, 4099) and got[:10] == b"\0" * 10
    # mmap fill: the checksum of the generator's stream of the same seed
    assert res[2] == oracle.c5_checksum(workloads.stream_bytes(5, 65536))


def test_c5_trace_shape():
    tr = workloads.c5_trace(workloads.C5_SMALL)
    assert len(tr) == 200
    assert tr.threads.min() >= 64 and tr.threads.max() <= 65536
    assert np.all(np.diff(tr.arrival_ns.astype(np.int64)) >= 0)
    live = np.arange(8)[None, :] < tr.n_ops[:, None]
    kinds = tr.ops["kind"][live]
    assert set(np.unique(kinds)) <= {0, 1, 2}
    pw = tr.ops[live & (tr.ops["kind"] == 1)]
    ends = np.sort(pw["out_off"]) + pw["len"][np.argsort(pw["out_off"])]
    assert np.all(np.sort(pw["out_off"])[1:] >= ends[:-1])          # disjoint pwrite ranges
    mm = tr.ops[live & (tr.ops["kind"] == 2)]
    assert np.all(mm["len"] % 4096 == 0) and mm["len"].min() >= 4096


def test_c5_parallel_replay_equals_the_sequential_one(tmp_path):
    """The multi-process replay the full-trace parity checks use gives the
    sequential replay's results and output file, byte for byte (requests are
    independent: read-only inputs, disjoint output ranges)."""
    tr = workloads.c5_trace(workloads.C5_SMALL).subset(np.arange(60))
    seq_path, par_path = str(tmp_path / "seq.bin"), str(tmp_path / "par.bin")
    fd = os.open(seq_path, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
    try:
        want = oracle.c5_trace(tr, fd)
    finally:
        os.close(fd)
    got = oracle.c5_trace_parallel(tr, par_path, procs=3)
    assert np.array_equal(got, want)
    assert open(par_path, "rb").read() == open(seq_path, "rb").read()


# ------------------------------------------------------------------------- C4

def test_c4_replay_closed_forms():
    p = dict(workloads.C4_SMALL, n_keys=512, n_requests=3000)
    tr = workloads.kv_trace(p)
    reps = oracle.c4_replay(tr)
    last_set = {}
    for j in range(len(tr)):
        k, op, r = int(tr.key_idx[j]), int(tr.op[j]), reps[j]
        assert r[4:8] == j.to_bytes(4, "little")                 # seq echoed
        if op == workloads.KV_SET:
            assert r == bytes([0x81, 0, 0, 0]) + j.to_bytes(4, "little")
            last_set[k] = j
        else:
            assert r[0] == 0x80 and r[1] == 0
            if k in last_set:                                    # the latest SET of the key
                js = last_set[k]
                want = workloads.stream_bytes(int(tr.vseed[js]), int(tr.vlen[js]))
            else:                                                # never SET: the preload value
                want = tr.value0(k)
            assert int.from_bytes(r[2:4], "little") == len(want) and r[8:] == want


def test_c4_unknown_key_and_get_only_trace():
    p = dict(workloads.C4_SMALL, n_keys=64, n_requests=200, get_frac=1.0)
    tr = workloads.kv_trace(p)
    reps = oracle.c4_replay(tr)
    for j in range(len(tr)):
        assert reps[j][8:] == tr.value0(int(tr.key_idx[j]))    # pure function of the key
    # a key that is not in the table: status 1, no value (hand-made datagram)
    import ctypes
    absent = bytes(16)
    assert absent not in {k.tobytes() for k in tr.keys}
    dgram = bytes([0, 0, 0, 0]) + (7).to_bytes(4, "little") + absent
    vals = np.zeros((len(tr.keys), 1024), np.uint8)
    vl = tr.vlen0.astype(np.uint16).copy()
    out = np.zeros(64, np.uint8)
    off = np.zeros(2, np.uint64)
    keys = np.ascontiguousarray(tr.keys)
    n = oracle._L().oracle_c4_replay(keys.ctypes.data, len(keys), vals.ctypes.data, vl.ctypes.data,
                                     ctypes.create_string_buffer(dgram, len(dgram)), 1, out.ctypes.data,
                                     off.ctypes.data)
    assert n == 8 and out[:8].tobytes() == bytes([0x80, 1, 0, 0, 7, 0, 0, 0])


def test_c4_zipf_and_mix():
    tr = workloads.kv_trace(workloads.C4_SMALL)
    frac_set = (tr.op == workloads.KV_SET).mean()
    assert 0.08 < frac_set < 0.12
    counts = np.bincount(tr.key_idx, minlength=len(tr.keys))
    assert counts[0] == counts.max()                              # rank 1 is the most popular key
    assert tr.vlen0.min() >= 64 and tr.vlen0.max() <= 1024


# ------------------------------------------------------------------------- C6

def _c6(tmp_path, data, perm, iters, name="c6.bin"):
    p = str(tmp_path / name)
    oracle.c6_permute(data, perm, iters, p)
    return np.frombuffer(open(p, "rb").read(), np.uint8)


def test_c6_rotation_is_a_gather(tmp_path):
    # perm[i] = i + 1 (mod 8192): one gather step moves every byte one place
    # towards the block start, so k steps rotate left by k
    data = np.arange(2 * 8192, dtype=np.uint64).astype(np.uint8)
    rot = ((np.arange(8192) + 1) % 8192).astype(np.uint16)
    for k in (0, 1, 5):
        got = _c6(tmp_path, data, rot, k).reshape(2, 8192)
        for b in range(2):
            assert np.array_equal(got[b], np.roll(data.reshape(2, 8192)[b], -k))


def test_c6_group_invariants(tmp_path):
    data, perm = workloads.c6_inputs(3)
    assert sorted(perm.tolist()) == list(range(8192))              # a bijection
    # cycle decomposition -> order of the permutation
    seen, lens = np.zeros(8192, bool), []
    for i in range(8192):
        if not seen[i]:
            n, j = 0, i
            while not seen[j]:
                seen[j] = True
                j = int(perm[j])
                n += 1
            lens.append(n)
    order = int(np.lcm.reduce(np.array(lens, dtype=np.int64)))
    if order < 10_000:
        assert np.array_equal(_c6(tmp_path, data, perm, order), data)   # pi^order = identity
    # composition: 3 steps then 4 steps == 7 steps
    a3 = _c6(tmp_path, data, perm, 3, "a3.bin")
    assert np.array_equal(_c6(tmp_path, a3, perm, 4, "a7.bin"), _c6(tmp_path, data, perm, 7, "b7.bin"))
    # a permutation keeps each block's multiset of bytes
    out = _c6(tmp_path, data, perm, 9).reshape(3, 8192)
    for b in range(3):
        assert np.array_equal(np.sort(out[b]), np.sort(data.reshape(3, 8192)[b]))
    # the identity permutation changes nothing
    ident = np.arange(8192, dtype=np.uint16)
    assert np.array_equal(_c6(tmp_path, data, ident, 11), data)
