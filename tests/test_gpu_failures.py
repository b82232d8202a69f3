"""Failure handling on the GPU without faulting it: a device wait that runs out
(nobody services the call) returns an error status the host reads, and the
context stays usable.  Failures are made on the host side only."""
import errno
import os
import threading

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NR_NOP = 0x7F00


@pytest.fixture(scope="module")
def G():
    import paper_1705_06965_b300 as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return G


def test_unserviced_call_times_out_and_context_recovers(G):
    # no service threads: until the host calls genesys_service, nothing answers
    with G.Context(device=0, no_threads=True, service_threads=1, deadline_ns=50_000_000,
                   staging_bytes=1 << 20) as ctx:
        with pytest.raises(G.GenesysError) as e:
            ctx.gpu_call(NR_NOP, [5], G.GRAN_GROUP, 64)
        assert e.value.code == G.EDEVICE
        assert ctx.stats()["requests"] == 1          # the drain answered the late request
        # with the host servicing while the kernel runs, the same call succeeds
        stop = threading.Event()

        def serve():
            while not stop.is_set():
                ctx.service(1_000_000)

        t = threading.Thread(target=serve)
        t.start()
        try:
            assert ctx.gpu_call(NR_NOP, [7], G.GRAN_GROUP, 64) == 7
            assert ctx.gpu_call(NR_NOP, [9], G.GRAN_ITEM, 1) == 9
        finally:
            stop.set()
            t.join()
        assert ctx.status() == [0] * G.ST_WORDS


def test_failed_syscall_is_a_result_not_a_fault(G):
    with G.Context(device=0, service_threads=1, staging_bytes=1 << 20) as ctx:
        assert ctx.gpu_call(17, [987654, 0, 16, 0]) == -errno.EBADF   # pread on a closed fd
        assert ctx.status()[G.ST_FAILED_CALLS] >= 0


def test_service_thread_restart_during_a_kernel(G, tmp_path):
    """A service thread is stopped and restarted (20 ms unserved) while a
    work-item-grain pwrite kernel runs: its calls wait, complete after the
    restart, and the file is exact."""
    import oracle
    import workloads
    n = 1 << 18
    with G.Context(device=0, service_threads=2, staging_bytes=n * 64 + (1 << 20), deadline_ns=5_000_000_000) as ctx:
        st = ctx.staging(n * 64)
        p = str(tmp_path / "r.bin")
        fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
        err = []

        def run():
            try:
                ctx.c2_pwrite(fd, n, G.GRAN_ITEM, 256, False, False, workloads.SEED_C2, st, n * 64)
            except Exception as e:  # reported below
                err.append(e)

        t = threading.Thread(target=run)
        t.start()
        for ring in (0, 1):
            ctx.service_restart(ring, pause_ns=20_000_000)
        # the watchdog probe works while the kernel runs (reads the rings'
        # producer positions on a non-blocking stream)
        stalled, pending = ctx.service_health(1_000_000_000)
        assert stalled == [] and pending >= 0
        t.join()
        os.close(fd)
        assert not err, err
        want = str(tmp_path / "w.bin")
        oracle.c2_pwrite(want, n, 1)
        assert open(p, "rb").read() == open(want, "rb").read()
        assert ctx.status() == [0] * G.ST_WORDS
