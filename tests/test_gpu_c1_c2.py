"""GPU parity: C1 (pread + byte histogram) and C2 (pwrite at every granularity,
ordering and blocking mode) against the CPU oracle, bit-exact; the strong
ordering visibility probe; the legality rules of Sec. 4.1.

All calls go through the C ABI (libgenesys.so) via the ctypes binding.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    import paper_1705_06965_b300 as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return G


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(device=0, service_threads=4, staging_bytes=320 << 20, deadline_ns=5_000_000_000)
    yield c
    c.close()


def _c1(ctx, G, path, nbytes, chunk, groups, threads, form):
    hist = torch.zeros(256, dtype=torch.int32, device="cuda")
    ctx.staging_reset()
    need = groups * chunk * (threads // 32 if form == G.FORM_WARP else 2)
    st = ctx.staging(need)
    fd = os.open(path, os.O_RDONLY)
    try:
        ctx.c1_histogram(fd, nbytes, hist.data_ptr(), st, need, chunk=chunk, groups=groups, threads=threads,
                         form=form)
    finally:
        os.close(fd)
    torch.cuda.synchronize()
    return hist.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("form", [0, 1, 2, 3])
def test_c1_full_config_bit_exact(ctx, G, form):
    """The C1 configuration: 4 MiB, 64 work-groups x 256 threads, 4 KiB preads."""
    p = workloads.c1_file()
    want = oracle.c1_histogram(p, 4096)
    got = _c1(ctx, G, p, 4 << 20, 4096, 64, 256, form)
    assert np.array_equal(got, want)
    assert ctx.status() == [0] * G.ST_WORDS


@pytest.mark.parametrize("nbytes,chunk,groups,threads", [
    (1, 4096, 64, 256),               # less than one chunk
    (4096 * 3 + 17, 4096, 64, 256),   # fewer chunks than groups, ragged tail
    (1 << 20, 16, 8, 32),             # tiny chunks: many calls per group
    ((1 << 20) + 123, 65536, 148, 1024),
    (6 << 20, 1 << 20, 5, 512),
])
@pytest.mark.parametrize("form", [0, 1, 2, 3])
def test_c1_shapes(ctx, G, tmp_path, nbytes, chunk, groups, threads, form):
    p = workloads.c1_file(str(tmp_path / "c1.bin"), nbytes, seed=nbytes)
    want = oracle.c1_histogram(p, chunk)
    got = _c1(ctx, G, p, nbytes, chunk, groups, threads, form)
    assert np.array_equal(got, want)


def test_c1_empty_and_errors(ctx, G, tmp_path):
    p = workloads.c1_file(str(tmp_path / "e.bin"), 0)
    assert _c1(ctx, G, p, 0, 4096, 4, 64, 0).sum() == 0
    hist = torch.zeros(256, dtype=torch.int32, device="cuda")
    st = ctx.staging(4096)
    with pytest.raises(G.GenesysError) as e:
        ctx.c1_histogram(3, 4096, hist.data_ptr(), st, 4096, chunk=4008, groups=1, threads=64)
    assert e.value.code == G.EINVAL        # chunk not a multiple of 16
    with pytest.raises(G.GenesysError) as e:
        ctx.c1_histogram(3, 4096, hist.data_ptr(), st, 4096, chunk=4096, groups=1, threads=64, form=4)
    assert e.value.code == G.EINVAL        # no such form
    with pytest.raises(G.GenesysError) as e:  # warp form: one chunk per warp in staging
        ctx.c1_histogram(3, 4096, hist.data_ptr(), st, 4096, chunk=4096, groups=1, threads=64, form=G.FORM_WARP)
    assert e.value.code == G.EINVAL
    # a file shorter than announced: preads return short, the histogram
    # covers the bytes that exist
    p2 = workloads.c1_file(str(tmp_path / "s.bin"), 5000, seed=3)
    got = _c1(ctx, G, p2, 64 * 4096, 4096, 4, 64, 0)
    assert np.array_equal(got, oracle.c1_histogram(p2, 4096))


def _c2(ctx, G, path, n, gran, bt, relaxed, nonblocking, seed=workloads.SEED_C2):
    ctx.staging_reset()
    st = ctx.staging(n * 64)
    fd = os.open(path, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
    try:
        ctx.c2_pwrite(fd, n, gran, bt, relaxed, nonblocking, seed, st, n * 64)
    finally:
        os.close(fd)
    with open(path, "rb") as f:
        return f.read()


COMBOS = [(g, r, nb) for g in range(4) for r in (False, True) for nb in (False, True) if not (g == 0 and r)]


@pytest.mark.parametrize("gran,relaxed,nonblocking", COMBOS)
@pytest.mark.parametrize("n,bt", [(1, 32), (4096 + 37, 256), (20000, 64), (1 << 14, 1024)])
def test_c2_combos_bit_exact(ctx, G, tmp_path, gran, relaxed, nonblocking, n, bt):
    want_path = str(tmp_path / "want.bin")
    group = {0: 1, 1: 32, 2: bt, 3: n}[gran]
    oracle.c2_pwrite(want_path, n, group)
    want = open(want_path, "rb").read()
    got = _c2(ctx, G, str(tmp_path / "got.bin"), n, gran, bt, relaxed, nonblocking)
    assert got == want
    assert ctx.status() == [0] * G.ST_WORDS


@pytest.mark.parametrize("gran", [0, 1, 2, 3])
def test_c2_full_size(ctx, G, gran):
    """2^20 threads (the top of the C2 sweep), work-group of 256."""
    n = 1 << 20
    d = workloads.scratch_dir("tests")
    want_path = os.path.join(d, "c2_want.bin")
    if not os.path.exists(want_path) or os.path.getsize(want_path) != n * 64:
        oracle.c2_pwrite(want_path, n, 256)
    got = _c2(ctx, G, os.path.join(d, "c2_got.bin"), n, gran, 256, gran != 0, False)
    assert got == open(want_path, "rb").read()


def test_c2_call_counts_and_latency(ctx, G, tmp_path):
    n = 8192
    for gran, calls in [(0, n), (1, n // 32), (2, n // 256), (3, 1)]:
        ctx.stats_reset()
        ctx.latency(clear=True)
        _c2(ctx, G, str(tmp_path / "x.bin"), n, gran, 256, gran != 0, False)
        st = ctx.stats()
        assert st["requests"] == calls, (gran, st)
        lat = ctx.latency(clear=True)
        assert len(lat) == calls and lat.min() > 0


def test_c2_illegal_item_relaxed(ctx, G, tmp_path):
    st = ctx.staging(64)
    with pytest.raises(G.GenesysError) as e:
        ctx.c2_pwrite(1, 1, 0, 32, True, False, 0, st, 64)
    assert e.value.code == G.EINVAL


@pytest.mark.parametrize("gran", [0, 1, 2, 3])
@pytest.mark.parametrize("n,bt", [(4096, 256), (20000, 1024)])
def test_strong_ordering_visibility(ctx, G, gran, n, bt):
    """Strong ordering: every store made before the call is visible to the CPU
    handler (Sec. 4.1).  Violations must be 0."""
    ctx.staging_reset()
    probe = ctx.staging(n * 8)
    ctx.host_view(probe, n * 8)[:] = 0
    viol = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.visibility_probe(n, gran, bt, False, 0xABCDEF, probe, viol.data_ptr())
    assert int(viol.item()) == 0


def test_relaxed_consumer_runs(ctx, G):
    """Relaxed consumer role has no barrier before the call: the check may see
    stores still in flight (allowed); it must complete without errors."""
    n = 1 << 16
    ctx.staging_reset()
    probe = ctx.staging(n * 8)
    ctx.host_view(probe, n * 8)[:] = 0
    viol = torch.zeros(1, dtype=torch.int64, device="cuda")
    for gran in (1, 2, 3):
        ctx.visibility_probe(n, gran, 256, True, 7, probe, viol.data_ptr())
    assert int(viol.item()) >= 0


@pytest.mark.parametrize("n_slots,threads,window", [(64, 1, 0), (256, 3, 0), (1024, 2, 50_000)])
def test_c2_small_slot_area_and_coalescing_window(G, tmp_path, n_slots, threads, window):
    """A slot area far smaller than the number of callers (claims probe and wait
    for slots to free up, rings wrap many times), and a coalescing window:
    the file is still the oracle's."""
    n = 1 << 14
    want_path = str(tmp_path / "want.bin")
    oracle.c2_pwrite(want_path, n, 1)
    with G.Context(device=0, n_slots=n_slots, service_threads=threads, coalesce_window_ns=window,
                   staging_bytes=(n * 64) + (1 << 20), deadline_ns=10_000_000_000) as c:
        for gran, relaxed, nb in [(0, False, False), (0, False, True), (1, True, True), (2, False, False)]:
            got = _c2(c, G, str(tmp_path / "got.bin"), n, gran, 256, relaxed, nb)
            assert got == open(want_path, "rb").read(), (gran, relaxed, nb)
        st = c.stats()
        assert st["failed"] == 0


def test_c2_every_combination_on_a_64_slot_area(G, tmp_path):
    """Every legal grain x ordering x blocking combination with 4,133 threads
    on a 64-slot area: callers outnumber slots 65 to 1, so work-item lanes wait
    for slots and lone callers find all 32 they try busy and wait for one; the
    files equal the oracle's and no wait runs out."""
    n = 4096 + 37
    with G.Context(device=0, n_slots=64, service_threads=2, staging_bytes=n * 64 + (1 << 20),
                   deadline_ns=10_000_000_000) as c:
        for gran, relaxed, nb in COMBOS:
            for bt in ((64, 256) if gran == 2 else (256,)):
                want_path = str(tmp_path / "want.bin")
                oracle.c2_pwrite(want_path, n, {0: 1, 1: 32, 2: bt, 3: n}[gran])
                got = _c2(c, G, str(tmp_path / "got.bin"), n, gran, bt, relaxed, nb)
                assert got == open(want_path, "rb").read(), (gran, bt, relaxed, nb)
                assert c.status() == [0] * G.ST_WORDS, (gran, bt, relaxed, nb)


@pytest.mark.parametrize("gran,bt", [(1, 256), (2, 64)])
def test_nonblocking_callers_pass_over_slots_still_in_flight(G, tmp_path, gran, bt):
    """Non-blocking warp and work-group pwrites of 2^20 threads on a context
    whose rings nobody serves until the kernel has ended (no service threads;
    the drain serves them afterwards).  Later blocks on an SM start from the
    slots of their hardware ids, whose previous requests are still unserved:
    they take other ready slots instead of waiting, so the kernel ends on its
    own (a caller that waited would run into the 2 s deadline), and the file
    is the oracle's."""
    n = 1 << 20
    group = {1: 32, 2: bt}[gran]
    want_path = str(tmp_path / "want.bin")
    oracle.c2_pwrite(want_path, n, group)
    with G.Context(device=0, no_threads=True, service_threads=2, staging_bytes=n * 64 + (1 << 20),
                   deadline_ns=2_000_000_000) as c:
        for relaxed in (False, True):
            got = _c2(c, G, str(tmp_path / "got.bin"), n, gran, bt, relaxed, True)
            assert got == open(want_path, "rb").read(), relaxed
            assert c.status() == [0] * G.ST_WORDS
        assert c.stats()["requests"] == 2 * n // group


def test_service_probe_leaves_the_context_usable(G, tmp_path):
    """genesys_service_probe publishes work-item pwrites from the host into
    the same slot area and rewrites the device-side claim state: kernels on
    the context afterwards still claim, complete and write exactly."""
    with G.Context(device=0, service_threads=2, n_slots=4096, staging_bytes=(1 << 20) * 64 + (1 << 20),
                   deadline_ns=5_000_000_000) as c:
        n = 1 << 14
        st = c.staging(n * 64 * 2)
        view = c.host_view(st, n * 64)
        view[:] = np.frombuffer(workloads.stream_bytes(5, n * 64), np.uint8)
        p = str(tmp_path / "probe.bin")
        fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        try:
            rate = c.service_probe(fd, st, 64, n)   # 4 rounds of the 4096-slot area
            assert rate > 0
        finally:
            os.close(fd)
        assert open(p, "rb").read() == workloads.stream_bytes(5, n * 64)
        for gran, bt in ((0, 256), (1, 256), (2, 64)):
            want_path = str(tmp_path / f"want_{gran}.bin")
            oracle.c2_pwrite(want_path, 20000, {0: 1, 1: 32, 2: bt}[gran])
            q = str(tmp_path / f"after_{gran}.bin")
            fd = os.open(q, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
            try:
                c.c2_pwrite(fd, 20000, gran, bt, False, False, workloads.SEED_C2, st + n * 64, 20000 * 64)
            finally:
                os.close(fd)
            assert open(q, "rb").read() == open(want_path, "rb").read()
        assert c.status() == [0] * G.ST_WORDS


@pytest.mark.parametrize("factor", [2, 3, 4, 8])
@pytest.mark.parametrize("nbytes,chunk,groups", [((1 << 20) + 123, 4096, 16), (4096 * 5 + 9, 4096, 4)])
def test_c1_batched_read_depths(ctx, G, tmp_path, factor, nbytes, chunk, groups):
    """The batched form keeps as many reads in flight per block as the staging
    holds (2..4): ragged files, fewer chunks than buffers, all equal the oracle."""
    p = workloads.c1_file(str(tmp_path / "d.bin"), nbytes, seed=factor)
    want = oracle.c1_histogram(p, chunk)
    hist = torch.zeros(256, dtype=torch.int32, device="cuda")
    ctx.staging_reset()
    need = groups * chunk * factor
    st = ctx.staging(need)
    fd = os.open(p, os.O_RDONLY)
    try:
        ctx.c1_histogram(fd, nbytes, hist.data_ptr(), st, need, chunk=chunk, groups=groups, threads=256,
                         form=G.FORM_BATCHED)
    finally:
        os.close(fd)
    assert np.array_equal(hist.cpu().numpy().view(np.uint32), want)
    assert ctx.status() == [0] * G.ST_WORDS
