"""The rest of the paper's implemented call set made from GPU code (Sec. 5,
Sec. 8.1: open, read, write, lseek, close, madvise beside pread/pwrite/mmap):
each call's effect is checked on the host."""
import errno
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SYS_read, SYS_write, SYS_open, SYS_close, SYS_lseek, SYS_madvise, SYS_getpid = 0, 1, 2, 3, 8, 28, 39
O_RDWR, O_CREAT = 0o2, 0o100


@pytest.fixture(scope="module")
def G():
    import paper_1705_06965_b300 as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return G


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(device=0, service_threads=2, staging_bytes=8 << 20)
    yield c
    c.close()


@pytest.mark.parametrize("gran,threads", [(0, 1), (1, 32), (2, 256)])
def test_open_write_lseek_read_close_from_gpu(G, ctx, tmp_path, gran, threads):
    ctx.staging_reset()
    path = str(tmp_path / "f.txt").encode() + b"\0"
    pbuf = ctx.staging(len(path))
    ctx.host_view(pbuf, len(path))[:] = np.frombuffer(path, np.uint8)
    fd = ctx.gpu_call(SYS_open, [pbuf, O_RDWR | O_CREAT, 0o644], gran, threads)
    assert fd >= 0
    msg = b"GPU system calls"
    wbuf = ctx.staging(64)
    ctx.host_view(wbuf, len(msg))[:] = np.frombuffer(msg, np.uint8)
    assert ctx.gpu_call(SYS_write, [fd, wbuf, len(msg)], gran, threads) == len(msg)
    assert ctx.gpu_call(SYS_lseek, [fd, 4, 0], gran, threads) == 4          # SEEK_SET
    rbuf = ctx.staging(64)
    assert ctx.gpu_call(SYS_read, [fd, rbuf, 64], gran, threads) == len(msg) - 4
    assert bytes(ctx.host_view(rbuf, len(msg) - 4)) == msg[4:]
    assert ctx.gpu_call(SYS_close, [fd], gran, threads) == 0
    assert ctx.gpu_call(SYS_close, [fd], gran, threads) == -errno.EBADF
    assert open(tmp_path / "f.txt", "rb").read() == msg


def test_madvise_and_getpid_from_gpu(G, ctx):
    ctx.staging_reset()
    buf = ctx.staging(1 << 20)
    page = (buf + 4095) & ~4095
    assert ctx.gpu_call(SYS_madvise, [page, 4096, 0]) == 0                   # MADV_NORMAL
    assert ctx.gpu_call(SYS_madvise, [page, 4096, 12345]) == -errno.EINVAL
    assert ctx.gpu_call(SYS_getpid) == os.getpid()
    assert ctx.gpu_call(200) == -errno.ENOSYS                               # not in the supported set


def test_link_pingpong_round_trip():
    """The host-link round trip under every blocking call: a GPU thread and a
    host thread exchange 2,000 flags; the time per round trip is positive and
    below the 10 us a PCIe round trip plus a polling host stays well under."""
    import paper_1705_06965_b300 as G
    ns = G.link_pingpong(0, rounds=2000)
    assert 100 < ns < 10_000, ns


def test_link_stream_reads_and_writes_pinned_memory():
    """The SMs' zero-copy streaming over the host link: the write form stores
    its pattern (word i = i, i >> 32, ~i, 0x5EED) into every 16-byte word of a
    256 MiB pinned buffer exactly once, and both directions move more than
    5 GB/s (a PCIe Gen6 x16 link carries about ten times that); misuse is
    refused."""
    import numpy as np
    import paper_1705_06965_b300 as G
    n = 256 << 20
    buf = torch.zeros(n // 4, dtype=torch.int32, pin_memory=True)
    w = G.link_stream(buf.data_ptr(), n, write=True, reps=1)
    words = buf.numpy().view(np.uint32).reshape(-1, 4)
    i = np.arange(len(words), dtype=np.uint64)
    assert np.array_equal(words[:, 0], (i & 0xFFFFFFFF).astype(np.uint32))
    assert np.array_equal(words[:, 1], (i >> 32).astype(np.uint32))
    assert np.array_equal(words[:, 2], (~i & 0xFFFFFFFF).astype(np.uint32))
    assert (words[:, 3] == 0x5EED).all()
    r = G.link_stream(buf.data_ptr(), n, write=False, reps=2)
    assert r > 5.0 and w > 5.0, (r, w)
    # both directions at once: the odd blocks write the second half (the same
    # pattern, counted from its start); the even blocks only read the first
    buf.zero_()
    b = G.link_stream(buf.data_ptr(), n, write=2, reps=1)
    half = len(words) // 2
    assert (words[:half] == 0).all()
    j = np.arange(half, dtype=np.uint64)
    assert np.array_equal(words[half:, 0], (j & 0xFFFFFFFF).astype(np.uint32))
    assert np.array_equal(words[half:, 2], (~j & 0xFFFFFFFF).astype(np.uint32))
    assert b > 5.0, b
    with pytest.raises(G.GenesysError) as e:
        G.link_stream(buf.data_ptr() + 8, 4096)                    # not 16-byte aligned
    assert e.value.code == G.EINVAL
    host = np.zeros(4096, np.uint8)                                # pageable, not mapped
    with pytest.raises(G.GenesysError) as e:
        G.link_stream(host.ctypes.data, 4096)
    assert e.value.code == G.EINVAL


@pytest.mark.parametrize("gran,bt", [(0, 256), (2, 128)])
def test_call_trace_joins_and_adds_up(gran, bt, tmp_path):
    """Trace of a pwrite kernel: one device record per call, each joined with
    its host record; the stages are non-negative within the clock
    calibration's error."""
    import paper_1705_06965_b300 as G
    import workloads
    n = 4096
    calls = n if gran == 0 else n // bt
    with G.Context(device=0, service_threads=2, staging_bytes=n * 64 + (1 << 20), trace=2 * n) as ctx:
        st = ctx.staging(n * 64)
        fd = os.open(str(tmp_path / "t.bin"), os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
        try:
            ctx.c2_pwrite(fd, n, gran, bt, gran != 0, False, workloads.SEED_C2, st, n * 64)
        finally:
            os.close(fd)
        dev, host, off = ctx.trace_read()
    assert len(dev) == calls and len(host) == calls
    b = G.trace_breakdown(dev, host, off)
    assert b["joined"] == calls
    slack = 20_000  # ns: calibration error and clock granularity
    for k in ("claim", "service", "total"):
        assert b[k]["p50_ns"] >= 0, b
    for k in ("queue", "delivery"):
        assert b[k]["p50_ns"] >= -slack, b
    # the host stages lie inside the call: pickup after publish, completion
    # before the result is seen (up to the calibration error)
    assert b["service"]["p99_ns"] <= b["total"]["p99_ns"] + slack, b


def test_handle_less_genesys_syscall_from_a_kernel_of_ones_own(G, ctx, tmp_path):
    """include/genesys_syscall.cuh: a kernel built apart from the library binds
    the context's device view and calls genesys_syscall(nr, ...) - one
    work-item pwrite per thread (the plain form), then a work-group getpid.
    The file holds every thread's record and every call returned its own
    result."""
    import ctypes
    import subprocess
    from paper_1705_06965_b300 import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = str(tmp_path / "syscall_demo.so")
    r = subprocess.run([build.nvcc(), *build.ARCH, "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-shared", "-cudart",
                        "shared", "-I", os.path.join(root, "include"),
                        os.path.join(root, "tests", "c_abi", "syscall_demo.cu"), "-o", so],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    demo = ctypes.CDLL(so)
    demo.syscall_demo.restype = ctypes.c_int
    demo.syscall_demo.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_void_p, ctypes.c_void_p]
    blocks, threads = 8, 128
    n = blocks * threads
    ctx.staging_reset()
    rec = ctx.staging(n * 64)
    want = np.random.default_rng(1705).integers(0, 256, n * 64, dtype=np.uint8)
    ctx.host_view(rec, n * 64)[:] = want
    item = torch.full((n,), -1, dtype=torch.int64, device="cuda:0")
    group = torch.zeros(blocks, dtype=torch.int64, device="cuda:0")
    path = str(tmp_path / "records.bin")
    fd = os.open(path, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
    try:
        view = ctx.device_view()
        rc = demo.syscall_demo(ctypes.addressof(view), fd, rec, blocks, threads, item.data_ptr(), group.data_ptr())
        ctx.drain()
    finally:
        os.close(fd)
    assert rc == 0
    assert bool((item.cpu() == 64).all())
    assert bool((group.cpu() == os.getpid()).all())
    assert np.array_equal(np.fromfile(path, np.uint8), want)
    assert not any(ctx.status())
