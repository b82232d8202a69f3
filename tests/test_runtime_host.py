"""Host-side runtime tests (no GPU).

The service threads, doorbell rings, slot protocol, request merging and error
paths are exercised with CPU threads standing in for GPU lanes
(genesys_emulate_call on a host-only context), the way the CUDA callers use
them.  Failures are made on the host: bad file descriptors, unsupported calls,
a stalled service (nobody polls) that makes the caller's deadline fire.
"""
import errno
import ctypes
import os
import re
import threading
import time

import numpy as np
import pytest

import paper_1705_06965_b300 as G
import workloads

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def test_library_exports_every_declared_symbol():
    L = G.lib()
    declared = set()
    for h in os.listdir(INCLUDE):
        if h.endswith(".h"):
            txt = open(os.path.join(INCLUDE, h)).read()
            declared |= set(re.findall(r"^(?:int|void|const char|uint32_t|uint64_t)\b[^;(]*?\b(genesys_\w+)\s*\(", txt, re.M))
    assert declared, "no declarations found"
    assert declared == set(G.EXPORTS), declared ^ set(G.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_config_defaults():
    cfg = G.Config()
    assert G.lib().genesys_config_default(cfg) == 0
    assert cfg.n_service_threads == 4 and cfg.coalesce_max == 64 and cfg.merge == 1
    assert cfg.device_deadline_ns == 2_000_000_000


def _ctx(**kw):
    kw.setdefault("host_only", True)
    kw.setdefault("service_threads", 2)
    kw.setdefault("staging_bytes", 1 << 20)
    kw.setdefault("n_slots", 256)
    kw.setdefault("deadline_ns", 2_000_000_000)
    return G.Context(**kw)


def test_nop_roundtrip_and_stats():
    with _ctx() as c:
        for v in (0, 1, 12345, 2**31 - 1, 2**40 + 7, -5 & ((1 << 64) - 1)):
            r = c.emulate_call(G.NR_NOP, [v])
            want = v if v < 2**63 else v - 2**64
            assert r == want
        st = c.stats()
        assert st["requests"] == 6 and st["by_op"]["internal"] == 6 and st["os_calls"] == 0


def test_pread_pwrite_through_protocol(tmp_path):
    p = str(tmp_path / "f.bin")
    data = workloads.stream_bytes(7, 4096)
    with _ctx() as c:
        buf = c.staging(8192)
        view = c.host_view(buf, 8192)
        view[:4096] = np.frombuffer(data, np.uint8)
        fd = os.open(p, os.O_CREAT | os.O_RDWR, 0o644)
        try:
            assert c.emulate_call(G.SYS_pwrite64, [fd, buf, 4096, 100]) == 4096
            assert c.emulate_call(G.SYS_pread64, [fd, buf + 4096, 4096, 100]) == 4096
            assert bytes(view[4096:]) == data
            # short read at end of file
            assert c.emulate_call(G.SYS_pread64, [fd, buf + 4096, 4096, 4000]) == 196
        finally:
            os.close(fd)
        with open(p, "rb") as f:
            f.seek(100)
            assert f.read() == data


def test_errors_are_returned_not_raised(tmp_path):
    with _ctx() as c:
        buf = c.staging(64)
        assert c.emulate_call(G.SYS_pread64, [987654, buf, 64, 0]) == -errno.EBADF
        assert c.emulate_call(200, [0]) == -errno.ENOSYS          # not in the supported set
        # a non-blocking failure is counted, never silently lost
        c.emulate_call(G.SYS_pwrite64, [987654, buf, 64, 0], flags=0)
        c.drain(2_000_000_000)
        st = c.stats()
        assert st["failed"] == 3 and st["nonblocking_failed"] == 1


def test_any_syscall_flag():
    with _ctx(any_syscall=True) as c:
        assert c.emulate_call(G.SYS_getpid) == os.getpid()
        assert c.emulate_call(102) == os.getuid()                  # SYS_getuid passes through


@pytest.mark.parametrize("merge", [True, False])
def test_concurrent_contiguous_pwrites_merge(tmp_path, merge):
    """Many emulated lanes write their 64-byte pieces; with merging the service
    issues fewer Linux calls, and the file is the same either way."""
    n = 4096
    p = str(tmp_path / "m.bin")
    want = workloads.stream_bytes(workloads.SEED_C2, n * 64)
    with _ctx(merge=merge, coalesce_window_ns=200_000, n_slots=1024) as c:
        buf = c.staging(n * 64)
        c.host_view(buf, n * 64)[:] = np.frombuffer(want, np.uint8)
        fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        errs = []

        def lane(t0, step):
            for gid in range(t0, n, step):
                r = c.emulate_call(G.SYS_pwrite64, [fd, buf + gid * 64, 64, gid * 64], flags=0)
                if r != 0:
                    errs.append(r)

        th = [threading.Thread(target=lane, args=(i, 8)) for i in range(8)]
        [t.start() for t in th]
        [t.join() for t in th]
        c.drain(5_000_000_000)
        os.close(fd)
        st = c.stats()
        assert not errs
        assert st["requests"] == n and st["failed"] == 0
        if merge:
            assert st["os_calls"] <= n
        else:
            assert st["os_calls"] == n
    assert open(p, "rb").read() == want


def test_ring_wraps_many_times():
    # 256 slots, 2 rings of 256 entries: 20k calls wrap each ring ~40 times
    with _ctx(n_slots=256) as c:
        errs = []

        def lane(k):
            for i in range(2500):
                if c.emulate_call(G.NR_NOP, [k * 100000 + i]) != k * 100000 + i:
                    errs.append(i)

        th = [threading.Thread(target=lane, args=(k,)) for k in range(8)]
        [t.start() for t in th]
        [t.join() for t in th]
        assert not errs
        assert c.stats()["requests"] == 20000


def test_no_threads_mode_is_driven_by_service():
    with _ctx(no_threads=True) as c:
        out = {}

        def caller():
            out["r"] = c.emulate_call(G.NR_NOP, [42])

        t = threading.Thread(target=caller)
        t.start()
        n = 0
        for _ in range(200):
            n += c.service(1_000_000)
            if n:
                break
        t.join()
        assert out["r"] == 42 and n == 1


def test_stalled_service_makes_the_caller_time_out():
    # nobody services the rings: the caller's bounded wait gives up
    with _ctx(no_threads=True, deadline_ns=50_000_000) as c:
        with pytest.raises(G.GenesysError) as e:
            c.emulate_call(G.NR_NOP, [1])
        assert e.value.code == G.ETIMEDOUT
        # the request is still published; a late service completes it and the
        # slot becomes reusable
        assert c.service(5_000_000) >= 1
        assert c.emulate_call(G.NR_NOP, [2], flags=0) == 0
        assert c.service(5_000_000) >= 1


def test_drain_waits_for_nonblocking_calls(tmp_path):
    p = str(tmp_path / "d.bin")
    with _ctx() as c:
        buf = c.staging(64 * 100)
        c.host_view(buf, 6400)[:] = 7
        fd = os.open(p, os.O_CREAT | os.O_RDWR, 0o644)
        for i in range(100):
            assert c.emulate_call(G.SYS_pwrite64, [fd, buf + 64 * i, 64, 64 * i], flags=0) == 0
        c.drain(5_000_000_000)
        os.close(fd)
    assert open(p, "rb").read() == b"\x07" * 6400


def test_staging_arena_bounds():
    with _ctx(staging_bytes=4096) as c:
        a = c.staging(1000)
        b = c.staging(1000)
        assert a % 256 == 0 and b % 256 == 0 and b - a == 1024
        with pytest.raises(G.GenesysError):
            c.staging(4096)
        c.staging_reset()
        assert c.staging(4096) == a


def test_bad_configs():
    with pytest.raises(G.GenesysError):
        G.Context(host_only=True, service_threads=0)
    with pytest.raises(G.GenesysError):
        G.Context(host_only=True, deadline_ns=0)


def test_host_only_context_cannot_launch():
    import ctypes
    with _ctx() as c:
        one = (ctypes.c_uint32 * 3)(1, 1, 1)
        rc = G.lib().genesys_launch(c.handle, ctypes.c_void_p(1), one, one, 0, None, 0, None)
        assert rc == G.EINVAL


@pytest.mark.parametrize("n_slots,threads,n", [(256, 2, 1000), (64, 3, 64 * 7 + 5)])
def test_service_probe_writes_the_file_and_keeps_state(tmp_path, n_slots, threads, n):
    """The service ceiling probe publishes work-item pwrites itself: the file
    must hold the payload, and the context's claim state must let later calls
    (emulated callers) reuse the same slots."""
    p = str(tmp_path / "probe.bin")
    payload = np.frombuffer(workloads.stream_bytes(11, 64 * n), np.uint8).copy()
    with _ctx(n_slots=n_slots, service_threads=threads) as c:
        fd = os.open(p, os.O_CREAT | os.O_RDWR | os.O_TRUNC, 0o644)
        try:
            rate = c.service_probe(fd, payload.ctypes.data, 64, n)
            assert rate > 0
            st = c.stats()
            assert st["requests"] == n and st["failed"] == 0
            for k in range(2 * n_slots):  # every slot is claimed again afterwards
                assert c.emulate_call(G.NR_NOP, [k]) == k
            c.drain()
        finally:
            os.close(fd)
    with open(p, "rb") as f:
        assert f.read() == payload.tobytes()


def test_service_probe_needs_threads():
    with _ctx(no_threads=True) as c:
        with pytest.raises(G.GenesysError):
            c.service_probe(0, 1, 64, 1)


@pytest.mark.parametrize("pattern", ["in_order", "runs_shuffled", "interleaved", "reversed"])
def test_one_batch_of_neighbours_becomes_one_call(tmp_path, pattern):
    """A batch's pwrites are put in file order before merging, whatever order
    they were published in: 64 neighbouring 64-byte pwrites published as one
    batch become one Linux call, and the file is right."""
    n = 64
    idx = np.arange(n)
    if pattern == "runs_shuffled":   # warps' runs arriving out of order
        idx = np.concatenate([idx[r * 8:(r + 1) * 8] for r in (5, 2, 7, 0, 3, 6, 1, 4)])
    elif pattern == "interleaved":   # two lanes' requests alternating: 0, 32, 1, 33, ...
        idx = np.stack([idx[:n // 2], idx[n // 2:]]).T.ravel()
    elif pattern == "reversed":
        idx = idx[::-1]
    assert sorted(idx.tolist()) == list(range(n))
    p = str(tmp_path / "o.bin")
    want = workloads.stream_bytes(3, n * 64)
    with _ctx(no_threads=True, service_threads=1, n_slots=256, coalesce_max=n) as c:
        buf = c.staging(n * 64)
        c.host_view(buf, n * 64)[:] = np.frombuffer(want, np.uint8)
        fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        try:
            for gid in idx.tolist():
                assert c.emulate_call(G.SYS_pwrite64, [fd, buf + gid * 64, 64, gid * 64], flags=0) == 0
            done = 0
            for _ in range(100):
                done += c.service(1_000_000)
                if done == n:
                    break
            st = c.stats()
        finally:
            os.close(fd)
    assert done == n and st["requests"] == n and st["failed"] == 0
    assert st["os_calls"] == 1, st
    assert open(p, "rb").read() == want


def test_c_abi_from_plain_c(tmp_path):
    """The boundary is a C ABI: a plain C program compiled against
    include/genesys.h and linked with libgenesys.so runs the request protocol
    in a host-only context (no Python in the loop)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.dirname(G.LIB_PATH)
    exe = str(tmp_path / "host_only_client")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c_abi", "host_only_client.c"), "-o", exe,
                           G.LIB_PATH, "-Wl,-rpath," + pkg])
    out = subprocess.run([exe, str(tmp_path / "scratch.bin")], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr + out.stdout
    assert out.stdout.startswith("ok requests=66")


def test_ring_choice_spreads_reads_and_groups_writes(tmp_path):
    """Doorbell rings of positional file calls (genesys_ring_of_file, compiled
    from the layout header by a plain C program): a round of 64 neighbouring
    4 KiB preads reaches at least 3 of 4 rings, so the service threads copy in
    parallel, while neighbouring pwrites of one 16 KiB block (64-byte calls)
    and of one 256 KiB region (64 KiB calls) stay in one ring, where they
    merge."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "ring_regions")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c_abi", "ring_regions.c"), "-o", exe])
    out = subprocess.run([exe, "4"], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    got = dict(kv.split("=") for kv in out.stdout.split())
    assert int(got["reads_min_rings"]) >= 3, got
    assert int(got["writes_max_rings"]) == 1 and int(got["big_writes_max_rings"]) == 1, got


def test_service_thread_restart_loses_no_request():
    """A service thread is stopped and restarted while emulated callers keep
    calling: requests published meanwhile wait in the ring and are carried out
    by the new thread, each exactly once (every NOP returns its own argument
    and the request count matches)."""
    with _ctx(n_slots=256, service_threads=2, deadline_ns=5_000_000_000) as c:
        errs, done = [], []
        stop = threading.Event()

        def lane(k):
            i = 0
            while not stop.is_set() or i < 200:
                v = k * 1_000_000 + i
                if c.emulate_call(G.NR_NOP, [v]) != v:
                    errs.append(v)
                i += 1
            done.append(i)

        th = [threading.Thread(target=lane, args=(k,)) for k in range(4)]
        [t.start() for t in th]
        for ring in (0, 1, 0):
            c.service_restart(ring, pause_ns=30_000_000)
        stop.set()
        [t.join() for t in th]
        c.drain()
        assert not errs
        assert c.stats()["requests"] == sum(done)


def test_service_pause_past_the_deadline_times_out_then_recovers():
    with _ctx(n_slots=64, service_threads=1, deadline_ns=50_000_000) as c:
        out = {}

        def caller():
            try:
                out["r"] = c.emulate_call(G.NR_NOP, [3])
            except G.GenesysError as e:
                out["e"] = e.code

        t = threading.Thread(target=caller)
        restart = threading.Thread(target=c.service_restart, args=(0, 300_000_000))
        restart.start()
        time.sleep(0.05)            # the ring is unserved now
        t.start()
        t.join()
        restart.join()
        assert out.get("e") == G.ETIMEDOUT
        c.drain()                   # the late request is still carried out
        assert c.emulate_call(G.NR_NOP, [4]) == 4
        assert c.stats()["requests"] == 2


def test_service_restart_rejects_bad_use():
    with _ctx(no_threads=True) as c:
        with pytest.raises(G.GenesysError):
            c.service_restart(0)
    with _ctx(service_threads=2) as c:
        with pytest.raises(G.GenesysError):
            c.service_restart(2)


def test_host_trace_and_service_cpu_time():
    """With a trace kept, every request gets a host record (pickup <= done),
    reading clears it, and the service threads' CPU time is reported."""
    with _ctx(trace=4096, service_threads=2) as c:
        for v in range(300):
            assert c.emulate_call(G.NR_NOP, [v]) == v
        dev, host, off = c.trace_read()
        assert len(dev) == 0 and off == 0          # no device side in a host-only context
        assert len(host) == 300
        assert np.all(host["t_done"] >= host["t_pickup"]) and np.all(host["t_pickup"] > 0)
        assert len({(int(a), int(b)) for a, b in zip(host["slot"], host["seq"])}) == 300
        _, host2, _ = c.trace_read()
        assert len(host2) == 0
        assert c.stats()["service_cpu_ns"] > 0
        c.stats_reset()
        assert c.stats()["service_cpu_ns"] < 50_000_000


def test_trace_needs_capacity():
    with _ctx() as c:
        with pytest.raises(G.GenesysError):
            c.trace_read()


def test_trace_breakdown_joins_and_skips_unknown_publish_times():
    dev = np.zeros(3, G.TRACE_DEV_DTYPE)
    host = np.zeros(2, G.TRACE_HOST_DTYPE)
    dev["slot"], dev["seq"] = [1, 2, 3], [7, 7, 7]
    dev["t_call"], dev["t_publish"], dev["t_done"] = [100, 100, 100], [150, 0, 150], [400, 500, 0]
    host["slot"], host["seq"] = [1, 2], [7, 7]
    host["t_pickup"], host["t_done"] = [1200, 1210], [1300, 1310]
    b = G.trace_breakdown(dev, host, 1000)          # host clock = device clock + 1000 ns
    assert b["joined"] == 2                          # slot 3 is non-blocking (no t_done) and has no host record
    assert b["claim"] == {"p50_ns": 50, "p99_ns": 50}   # only the record with a publish time
    assert b["queue"]["p50_ns"] == 1200 - (150 + 1000)
    assert b["service"]["p50_ns"] == 100
    assert b["total"]["p99_ns"] <= 400
    dev["gran"] = [0, 2, 2]
    by = G.latency_by_gran(dev)
    assert by == {"work-item": {"calls": 1, "p50_ns": 300, "p99_ns": 300},
                  "work-group": {"calls": 1, "p50_ns": 400, "p99_ns": 400}}


def test_merged_preads_split_a_short_read_correctly(tmp_path):
    """Coalescing must not change any call's result (Sec. 4.2): eight 64-byte
    preads that continue each other merge into one Linux call; the file ends
    inside the fifth, so the results are 64, 64, 64, 64, 16, 0, 0, 0 - what
    each call alone would have returned - and the bytes land where each asked.
    The merged call came back short, so the three requests past its end are
    made again as calls of their own (each then returns 0 at end of file)."""
    p = str(tmp_path / "short.bin")
    data = workloads.stream_bytes(21, 4 * 64 + 16)
    open(p, "wb").write(data)
    with _ctx(no_threads=True, service_threads=1, n_slots=64, coalesce_max=64) as c:
        buf = c.staging(8 * 64)
        view = c.host_view(buf, 8 * 64)
        view[:] = 0xAA
        fd = os.open(p, os.O_RDONLY)
        try:
            threads, results = [], [None] * 8

            def call(i):
                results[i] = c.emulate_call(G.SYS_pread64, [fd, buf + 64 * i, 64, 64 * i])

            for i in range(8):
                t = threading.Thread(target=call, args=(i,))
                t.start()
                threads.append(t)
            time.sleep(0.2)        # all eight published before the one service pass
            served = 0
            for _ in range(200):
                served += c.service(1_000_000)
                if served >= 8:
                    break
            [t.join() for t in threads]
            st = c.stats()
            got = bytes(view)  # staging memory lives as long as the context
        finally:
            os.close(fd)
    assert results == [64, 64, 64, 64, 16, 0, 0, 0], results
    assert st["os_calls"] == 1 + 3, st
    assert got[:4 * 64 + 16] == data
    assert got[4 * 64 + 16:] == b"\xaa" * (8 * 64 - 4 * 64 - 16)


def _serve_concurrent(c, n, call):
    """Publish n emulated calls from n threads, then serve them as one pass of
    a NO_THREADS context; returns the results."""
    threads, results = [], [None] * n

    def run(i):
        results[i] = call(i)

    for i in range(n):
        t = threading.Thread(target=run, args=(i,))
        t.start()
        threads.append(t)
    time.sleep(0.2)        # all published before the one service pass
    served = 0
    for _ in range(200):
        served += c.service(1_000_000)
        if served >= n:
            break
    [t.join() for t in threads]
    return results


def test_merged_pwritev_with_a_bad_middle_buffer_gives_each_its_own_result(tmp_path):
    """Eight 64-byte pwrites that continue each other in the file, from
    scattered buffers, merge into one pwritev; the fourth request's buffer is
    not mapped.  Linux stops the merged call at that buffer and returns the
    bytes written before it: the first three requests keep 64, the fourth
    (made again alone) gets -EFAULT and the last four, made again alone, write
    their bytes and get 64 - what separate calls would have done."""
    p = str(tmp_path / "bad.bin")
    n, bad = 8, 3
    pieces = [workloads.stream_bytes(200 + i, 64) for i in range(n)]
    with _ctx(no_threads=True, service_threads=1, n_slots=64, coalesce_max=64) as c:
        buf = c.staging(n * 64)
        view = c.host_view(buf, n * 64)
        for i in range(n):  # piece i sits in buffer slot n-1-i (not neighbours: a vector call)
            view[(n - 1 - i) * 64:(n - i) * 64] = np.frombuffer(pieces[i], np.uint8)
        fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        try:
            def call(i):
                addr = 0x1000 if i == bad else buf + (n - 1 - i) * 64   # page 1: never mapped
                return c.emulate_call(G.SYS_pwrite64, [fd, addr, 64, 64 * i])
            results = _serve_concurrent(c, n, call)
            st = c.stats()
        finally:
            os.close(fd)
    assert results == [64, 64, 64, -errno.EFAULT, 64, 64, 64, 64], results
    assert st["os_calls"] == 1 + (n - bad), st
    data = open(p, "rb").read()
    assert data == b"".join(pieces[:bad]) + b"\0" * 64 + b"".join(pieces[bad + 1:])


def test_pread_cap_is_a_checked_build_knob():
    """genesys_check_pread_cap exists in every build but caps preads only in
    the checked one; elsewhere it is refused."""
    with _ctx() as c:
        with pytest.raises(G.GenesysError) as e:
            c.pread_cap(1000)
        assert e.value.code == G.EINVAL


def test_pread_cap_makes_short_reads_in_the_checked_build(tmp_path):
    """Checked build, preads capped at 100 bytes: a lone 1,000-byte pread
    returns 100; eight 64-byte preads that continue each other merge into one
    capped call of 100 bytes, so the first gets 64, the second the 36 that
    call covered (a short read), and the other six, made again alone, 64
    each; every byte lands where its request asked."""
    import subprocess
    import sys
    from paper_1705_06965_b300 import build
    build.build(device_checks=True)
    path = str(tmp_path / "cap.bin")
    open(path, "wb").write(workloads.stream_bytes(31, 4096))
    code = (
        "import os, threading, time, sys\n"
        "sys.path.insert(0, 'tests')\n"
        "import paper_1705_06965_b300 as G\n"
        "from test_runtime_host import _ctx, _serve_concurrent\n"
        "assert G.LIB_PATH.endswith('libgenesys_checked.so')\n"
        f"path = {path!r}\n"
        "data = open(path, 'rb').read()\n"
        "fd = os.open(path, os.O_RDONLY)\n"
        "with _ctx(service_threads=1) as c:\n"
        "    c.pread_cap(100)\n"
        "    b = c.staging(1000)\n"
        "    assert c.emulate_call(G.SYS_pread64, [fd, b, 1000, 5]) == 100\n"
        "    assert bytes(c.host_view(b, 100)) == data[5:105]\n"
        "with _ctx(no_threads=True, service_threads=1, n_slots=64, coalesce_max=64) as c:\n"
        "    c.pread_cap(100)\n"
        "    b = c.staging(512)\n"
        "    r = _serve_concurrent(c, 8, lambda i: c.emulate_call(G.SYS_pread64, [fd, b + 64 * i, 64, 64 * i]))\n"
        "    assert r == [64, 36] + [64] * 6, r\n"
        "    got = bytes(c.host_view(b, 512))\n"
        "    assert got[:100] == data[:100] and got[128:512] == data[128:512]\n"
        "    assert c.stats()['os_calls'] == 7\n"
        "os.close(fd)\n"
        "print('ok')\n")
    env = dict(os.environ, GENESYS_LIBRARY="checked")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_merged_pwrites_with_scattered_buffers_use_one_vector_call(tmp_path):
    """Neighbouring file ranges whose buffers are not neighbours merge into one
    pwritev; the file is right."""
    p = str(tmp_path / "v.bin")
    n = 16
    pieces = [workloads.stream_bytes(100 + i, 64) for i in range(n)]
    with _ctx(no_threads=True, service_threads=1, n_slots=64, coalesce_max=64) as c:
        buf = c.staging(n * 64)
        view = c.host_view(buf, n * 64)
        for i in range(n):  # piece i sits in buffer slot n-1-i
            view[(n - 1 - i) * 64:(n - i) * 64] = np.frombuffer(pieces[i], np.uint8)
        fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        try:
            for i in range(n):
                assert c.emulate_call(G.SYS_pwrite64, [fd, buf + (n - 1 - i) * 64, 64, 64 * i], flags=0) == 0
            served = 0
            for _ in range(100):
                served += c.service(1_000_000)
                if served >= n:
                    break
            st = c.stats()
        finally:
            os.close(fd)
    assert st["requests"] == n and st["os_calls"] == 1 and st["failed"] == 0
    assert open(p, "rb").read() == b"".join(pieces)


def test_binding_and_library_agree_on_struct_sizes():
    L = G.lib()  # loading already refuses a mismatch; check the values and the unknown case
    assert int(L.genesys_sizeof(0)) == ctypes.sizeof(G.Config)
    assert int(L.genesys_sizeof(1)) == ctypes.sizeof(G.Stats)
    assert int(L.genesys_sizeof(4)) == G.TRACE_DEV_DTYPE.itemsize == 40
    assert int(L.genesys_sizeof(5)) == G.TRACE_HOST_DTYPE.itemsize == 24
    assert int(L.genesys_sizeof(99)) == 0
    # the device view as raw bytes (for kernels of one's own), filled in
    with _ctx(n_slots=4096) as c:
        view = c.device_view()
        assert len(view) == int(L.genesys_sizeof(G.SIZEOF_DEV)) > 0
        assert any(view.raw)


def test_checked_build_host_protocol_checker(tmp_path):
    """The checked build also checks, on the host, that every slot's requests
    reach the service numbered 1, 2, 3, ...: concurrent emulated callers over
    a small slot area (every slot reused many times) give no protocol error."""
    import subprocess
    import sys
    from paper_1705_06965_b300 import build
    build.build(device_checks=True)
    code = (
        "import threading, paper_1705_06965_b300 as G\n"
        "assert G.LIB_PATH.endswith('libgenesys_checked.so')\n"
        "c = G.Context(host_only=True, service_threads=2, n_slots=64, staging_bytes=1 << 20)\n"
        "errs = []\n"
        "def lane(k):\n"
        "    for i in range(500):\n"
        "        if c.emulate_call(G.NR_NOP, [k * 10000 + i]) != k * 10000 + i: errs.append(i)\n"
        "th = [threading.Thread(target=lane, args=(k,)) for k in range(6)]\n"
        "[t.start() for t in th]; [t.join() for t in th]\n"
        "st = c.stats(); c.close()\n"
        "assert not errs and st['requests'] == 3000, (errs[:3], st['requests'])\n"
        "assert st['protocol_errors'] == 0, st['protocol_errors']\n"
        "print('ok')\n")
    env = dict(os.environ, GENESYS_LIBRARY="checked")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_every_entry_point_rejects_null_arguments():
    """The C ABI returns GENESYS_EINVAL for NULL contexts and pointers - no
    entry point touches CUDA or dereferences anything before checking
    (genesys_shutdown(NULL) is a no-op returning 0)."""
    L = G.lib()
    res = {}
    def t(name, *args):
        f = getattr(L, name)
        try:
            res[name] = f(*args)
        except Exception as e:
            res[name] = repr(e)
    t("genesys_config_default", None)
    t("genesys_init", None, 0, None)
    t("genesys_shutdown", None)
    t("genesys_device_view", None, None)
    t("genesys_launch", None, None, None, None, 0, None, 0, None)
    t("genesys_service", None, 0)
    t("genesys_drain", None, 0)
    t("genesys_stats_get", None, None)
    t("genesys_stats_reset", None)
    t("genesys_status", None, None, 0)
    t("genesys_latency", None, None, 0, None, 0)
    t("genesys_staging_reset", None)
    t("genesys_emulate_call", None, 0, None, 0, None)
    t("genesys_c1_histogram", None, 0, 0, 0, 0, 0, 0, None, 0, None, None)
    t("genesys_c2_pwrite", None, 0, 0, 0, 0, 0, 0, 0, None, 0, None)
    t("genesys_visibility_probe", None, 0, 0, 0, 0, 0, None, None, None)
    t("genesys_last_launch_ms", None, None)
    t("genesys_c3_wordcount", None, None, None, 0, None, None, 0, 0, 0, 0, 0, None, 0, None, None)
    t("genesys_c3_wordcount_noalloc", None, None, None, 0, None, None, 0, 0, 0, 0, 0, None, 0, None, None)
    t("genesys_serve_config_default", None)
    t("genesys_reclaim", None)
    t("genesys_mmap_reserve", None, None, 0)
    t("genesys_kv_start", None, None, None, None, 0, 0, 0, 0, 0, 0, None)
    t("genesys_kv_stop", None, 0, None)
    t("genesys_kv_value", None, 0, None)
    t("genesys_kv_client", None, None, 0, None, 0, 0, 0, None, None, None, None)
    t("genesys_c6_permute", None, 0, None, None, 0, 0, 0, 0, None, 0, None)
    t("genesys_gpu_call", None, 0, None, 0, 0, None, None)
    t("genesys_echo_start", None, 0, 0, 0, 0, 0, 0, 0, None)
    t("genesys_echo_stop", None, 0, None)
    t("genesys_echo_client", 0, 0, 0, 0, 0, 0, 0, 0, 0, None)
    t("genesys_service_probe", None, 0, None, 0, 0, None)
    t("genesys_link_pingpong", 0, 0, 0, None)
    t("genesys_link_stream", 0, None, 0, 0, 0, 0, 0, None)
    t("genesys_service_restart", None, 0, 0)
    t("genesys_trace_read", None, None, 0, None, None, 0, None, None)
    t("genesys_c5_serve", None, None, 0, None, 0, 0, None, None, None, None)
    t("genesys_stats", None, None)
    t("genesys_graph_launches", None, None)
    t("genesys_check_pread_cap", None, 0)
    t("genesys_kv_received", None, None, 0)
    assert res.pop("genesys_shutdown") == 0
    assert all(v == G.EINVAL for v in res.values()), res
    assert len(res) >= 35


def test_service_health_reports_an_unserved_ring():
    """The watchdog probe: requests waiting in a ring nobody services for
    longer than stall_ns are reported; once serviced, the ring is healthy."""
    with _ctx(no_threads=True, service_threads=2, n_slots=512) as c:
        assert c.service_health(1_000_000) == ([], 0)
        for v in range(40):
            assert c.emulate_call(G.NR_NOP, [v], flags=0) == 0    # non-blocking: published, not served
        time.sleep(0.02)
        stalled, pending = c.service_health(10_000_000)
        assert pending == 40 and stalled, (stalled, pending)
        n = 0
        for _ in range(100):
            n += c.service(1_000_000)
            if n == 40:
                break
        assert c.service_health(10_000_000) == ([], 0)


def test_service_health_sees_a_paused_thread():
    with _ctx(service_threads=1, n_slots=64, deadline_ns=5_000_000_000) as c:
        assert c.emulate_call(G.NR_NOP, [1]) == 1
        restart = threading.Thread(target=c.service_restart, args=(0, 300_000_000))
        restart.start()
        time.sleep(0.05)
        caller = threading.Thread(target=c.emulate_call, args=(G.NR_NOP, [2]))
        caller.start()
        time.sleep(0.1)
        stalled, pending = c.service_health(50_000_000)
        assert stalled == [0] and pending == 1
        restart.join()
        caller.join()
        assert c.service_health(50_000_000) == ([], 0)


@pytest.mark.parametrize("src", ["user_kernel.cu", "syscall_demo.cu", "launch_demo.cu"])
def test_a_user_kernel_compiles_against_the_headers(tmp_path, src):
    """The device headers are usable from a user's own kernel: a pread kernel
    through genesys::call, a kernel of the handle-less genesys_syscall and the
    launch demo (graph relaunch, kernel-grain sites) compile for sm_103a with
    nothing but include/ (not run here)."""
    import shutil
    import subprocess
    from paper_1705_06965_b300 import build
    nvcc = build.nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([nvcc, *build.ARCH, "-std=c++17", "-c", "-I", os.path.join(root, "include"),
                        os.path.join(root, "tests", "c_abi", src), "-o", str(tmp_path / "u.o")],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


def _open_fds():
    return len(os.listdir("/proc/self/fd"))


def test_no_cxx_exception_crosses_the_c_abi():
    """A request count no host vector can hold comes back as an error code
    (the library catches the C++ exception at the entry point), and the
    sockets the call would have opened are not leaked."""
    L = G.lib()
    reqs = np.zeros(64, np.uint8)
    off = np.zeros(2, np.uint64)
    arr = np.zeros(1, np.uint64)
    out8 = np.zeros(64, np.uint8)
    rl = np.zeros(1, np.uint32)
    lat = np.zeros(1, np.uint64)
    stats = np.zeros(6, np.uint64)
    before = _open_fds()
    rc = L.genesys_kv_client(reqs.ctypes.data, off.ctypes.data, 1 << 62, arr.ctypes.data, 47000, 4, 1_000_000,
                             out8.ctypes.data, rl.ctypes.data, lat.ctypes.data, stats.ctypes.data)
    assert rc == G.EINVAL
    assert "genesys_kv_client" in L.genesys_last_error().decode()
    assert _open_fds() == before


_THREADS_CANNOT_START = r'''
import resource
import paper_1705_06965_b300 as G
G.lib()
vm = [int(l.split()[1]) * 1024 for l in open("/proc/self/status") if l.startswith("VmSize:")][0]
# room for the context's memory but not for 64 thread stacks
resource.setrlimit(resource.RLIMIT_AS, (vm + (96 << 20), resource.RLIM_INFINITY))
try:
    G.Context(host_only=True, service_threads=64, n_slots=32, staging_bytes=0)
    print("started")
except G.GenesysError as e:
    print("code", e.code)
resource.setrlimit(resource.RLIMIT_AS, (resource.RLIM_INFINITY, resource.RLIM_INFINITY))
with G.Context(host_only=True, service_threads=2, n_slots=32, staging_bytes=0) as c:
    print("after", c.emulate_call(G.SYS_getpid))
'''


def test_service_threads_that_cannot_start_are_an_error_not_an_abort():
    """genesys_init with an address-space limit that leaves no room for the
    service threads' stacks: the thread that fails to start becomes
    GENESYS_ENOMEM (the started ones are stopped and joined, the memory given
    back), and the process goes on to open a context normally."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _THREADS_CANNOT_START], cwd=root, capture_output=True, text=True,
                       timeout=120, env=dict(os.environ, PYTHONPATH=root))
    assert r.returncode == 0, r.stdout + r.stderr
    out = r.stdout.split("\n")
    if "started" in out:
        pytest.skip("the address-space limit did not stop the threads here")
    assert f"code {G.ENOMEM}" in out, r.stdout
    assert any(ln.startswith("after ") and int(ln.split()[1]) > 0 for ln in out), r.stdout


def test_service_probe_in_warp_interleaved_order(tmp_path):
    """genesys_service_probe_order: with the doorbells of 32-call runs rung
    eight runs apart, every call still lands (the file is the payload), and a
    batch no longer holds a run's neighbours, so the merged calls cover one
    run each - as with GPU work-items, whose batches merge about a warp."""
    n = 1 << 16
    fd = os.open(str(tmp_path / "o.bin"), os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o600)
    try:
        with _ctx(service_threads=2, coalesce_max=64, n_slots=65536, staging_bytes=n * 64 + 4096) as c:
            p = c.staging(n * 64)
            want = np.random.default_rng(11).integers(0, 256, n * 64, dtype=np.uint8)
            c.host_view(p, n * 64)[:] = want
            c.stats_reset()
            assert c.service_probe(fd, p, 64, n, run=32, stride=8) > 0
            st = c.stats()
            with pytest.raises(G.GenesysError):
                c.service_probe(fd, p, 64, n, run=0, stride=8)
        got = np.fromfile(str(tmp_path / "o.bin"), np.uint8)
    finally:
        os.close(fd)
    assert np.array_equal(got, want)
    assert st["requests"] == n and st["failed"] == 0
    assert st["requests"] / st["os_calls"] <= 32.0
