"""GPU parity for C5 (serving a trace of syscall-issuing kernels): every
request's results (pread checksums, pwrite byte counts, mmap-fill checksums)
and the output file equal the CPU oracle's, bit-exact; each request's result
is the same when it runs alone (one request on the GPU at a time) and in the
mix (up to 32 overlapping, admitted as budgets free up), with and without
CUDA-graph relaunch, with preads landing in pinned staging or in HBM, and
with one persistent executor kernel serving every request instead of a
kernel per request; the full 10,000-request trace in both serving forms."""
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
    c = G.Context(device=0, service_threads=8, staging_bytes=256 << 20, deadline_ns=10_000_000_000)
    yield c
    c.close()


@pytest.fixture(scope="module")
def trace():
    return workloads.c5_trace(workloads.C5_SMALL)


@pytest.fixture(scope="module")
def want(trace, tmp_path_factory):
    p = str(tmp_path_factory.mktemp("c5") / "oracle_out.bin")
    fd = os.open(p, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
    try:
        res = oracle.c5_trace(trace, fd)
    finally:
        os.close(fd)
    return res, open(p, "rb").read()


def serve(ctx, tr, out_path, **cfg):
    in_fds = [os.open(p, os.O_RDONLY) for p in tr.in_paths]
    out_fd = os.open(out_path, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
    try:
        res, lat, st = ctx.c5_serve(tr.arrival_ns, tr.threads, tr.n_ops, tr.ops, in_fds, out_fd, **cfg)
    finally:
        for fd in in_fds:
            os.close(fd)
        os.close(out_fd)
    return res, lat, st, open(out_path, "rb").read()


def _mask(tr):
    return np.arange(8)[None, :] < tr.n_ops[:, None]


def test_c5_mix_matches_oracle(ctx, trace, want, tmp_path):
    res, lat, st, out = serve(ctx, trace, str(tmp_path / "mix.bin"), max_inflight=32)
    m = _mask(trace)
    assert np.array_equal(res[m], want[0][m])
    assert out == want[1]
    assert st["requests"] == len(trace) and st["max_inflight"] > 1
    assert np.all(lat > 0)


def test_c5_alone_equals_mix(ctx, trace, want, tmp_path):
    alone, _, st1, out1 = serve(ctx, trace, str(tmp_path / "alone.bin"), max_inflight=1)
    mix, _, st2, out2 = serve(ctx, trace, str(tmp_path / "mix2.bin"), max_inflight=32, honor_arrivals=0)
    m = _mask(trace)
    assert st1["max_inflight"] == 1
    assert np.array_equal(alone[m], mix[m])
    assert np.array_equal(alone[m], want[0][m])
    assert out1 == out2 == want[1]


@pytest.mark.parametrize("use_graphs,pread_to_hbm,min_part", [(0, 0, 16384), (1, 1, 16384), (1, 0, 4096),
                                                              (1, 1, 1 << 20)])
def test_c5_variants(ctx, trace, want, tmp_path, use_graphs, pread_to_hbm, min_part):
    sub = trace.subset(np.arange(60))
    res, _, st, out = serve(ctx, sub, str(tmp_path / "v.bin"), max_inflight=16, use_graphs=use_graphs,
                            pread_to_hbm=pread_to_hbm, min_part=min_part, honor_arrivals=0)
    m = _mask(sub)
    assert np.array_equal(res[m], want[0][:60][m])
    if use_graphs:
        assert st["graph_launches"] == 60


def test_c5_budgets_throttle_admission(ctx, trace, want, tmp_path):
    # a tight staging budget admits fewer requests at a time; results unchanged
    sub = trace.subset(np.arange(40))
    res, _, st, _ = serve(ctx, sub, str(tmp_path / "b.bin"), max_inflight=32, staging_budget=4 << 20,
                          slot_budget=600, honor_arrivals=0)
    m = _mask(sub)
    assert np.array_equal(res[m], want[0][:40][m])


def test_c5_rejects_oversized_request(ctx, G, trace, tmp_path):
    rw = np.where(((trace.ops["kind"] < 2) & _mask(trace)).any(axis=1))[0][:5]
    sub = trace.subset(rw)
    with pytest.raises(G.GenesysError) as e:
        serve(ctx, sub, str(tmp_path / "x.bin"), staging_budget=16)
    assert e.value.code == G.EINVAL


@pytest.mark.parametrize("max_inflight", [1, 32])
def test_c5_persistent_executor_matches_oracle(ctx, trace, want, tmp_path, max_inflight):
    """One executor kernel serves the whole trace (requests admitted as
    budgets free up, their blocks taken from a ring by the executor's
    blocks): the same results and file as the oracle, alone and in the mix."""
    res, lat, st, out = serve(ctx, trace, str(tmp_path / "p.bin"), persistent=1, max_inflight=max_inflight,
                              honor_arrivals=0)
    m = _mask(trace)
    assert np.array_equal(res[m], want[0][m])
    assert out == want[1]
    assert st["requests"] == len(trace) and st["graph_launches"] == 0 and np.all(lat > 0)
    assert st["max_inflight"] == max_inflight


def test_c5_persistent_executor_with_few_blocks_and_hbm_landing(ctx, trace, want, tmp_path):
    """Fewer executor blocks than a large request has blocks (a request's
    blocks then run one after another on the same executor blocks, and its
    kernel-grain mmap and munmap still meet), preads landing in HBM."""
    sub = trace.subset(np.arange(60))
    res, _, st, _ = serve(ctx, sub, str(tmp_path / "pf.bin"), persistent=1, persistent_blocks=3, max_inflight=8,
                          pread_to_hbm=1, honor_arrivals=0)
    m = _mask(sub)
    assert np.array_equal(res[m], want[0][:60][m])


@pytest.fixture(scope="module")
def full(tmp_path_factory):
    """The full 10,000-request trace and the oracle's replay of every request,
    one at a time (shared among host processes: requests are independent)."""
    tr = workloads.c5_trace(workloads.C5_FULL)
    ref_path = str(tmp_path_factory.mktemp("c5full") / "ref.bin")
    return tr, oracle.c5_trace_parallel(tr, ref_path), open(ref_path, "rb").read()


@pytest.mark.parametrize("form", [{}, {"persistent": 1}], ids=["kernel_per_request", "persistent_executor"])
def test_c5_full_trace_equals_oracle(G, full, tmp_path, form):
    """The full trace served the way the benchmark serves it (its context and
    serving settings: 128 in flight on 128 streams, 256 MiB staging and HBM
    budgets, 12 service threads; arrivals honoured; graph relaunch or the
    persistent executor): every request's results and the whole output file
    equal the oracle's."""
    import bench
    tr, want, ref = full
    with G.Context(device=0, service_threads=bench.C5_SERVICE_THREADS, staging_bytes=512 << 20,
                   deadline_ns=10_000_000_000) as c:
        res, lat, st, out = serve(c, tr, str(tmp_path / "full.bin"), **bench.C5_SERVE, **form)
    assert st["requests"] == len(tr) and np.all(lat > 0)
    assert st["max_inflight"] > 64
    bad = np.where(((res != want) & _mask(tr)).any(axis=1))[0]
    assert len(bad) == 0, (len(bad), bad[:5])
    assert out == ref
