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
