"""The allocation-free wordcount entry point (genesys_c3_wordcount_noalloc).

It serves callers that cannot allocate device memory while they run (a fixed
device footprint after start-up, or no tolerance for the device-wide
synchronisation a cudaMalloc/cudaFree can cause): its scratch is a fixed
file-scope device array instead of cudaMalloc'd memory.  This file is
collected last so that a run stopping at the first failure has run every other
test first; it also passes alone in a fresh process.

The test calls the new entry point through the C ABI twice in a row and checks
each result against genesys_c3_wordcount on the same inputs and against the
generator's recorded per-query counts, the ground truth the oracle is pinned
to (integer counts: the tolerance is exact equality, as in every wordcount
test).  The caller's current CUDA device is the same after the first call,
which sets up the array's address, as before it.
"""
import ctypes
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pack_queries(queries):
    q = np.zeros((len(queries), 16), np.uint8)
    ql = np.zeros(len(queries), np.uint8)
    for i, s in enumerate(queries):
        q[i, :len(s)] = np.frombuffer(s, np.uint8)
        ql[i] = len(s)
    return q, ql


def test_noalloc_wordcount_matches_allocating_entry_point():
    import paper_1705_06965_b300 as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = G.lib()
    corpus = workloads.corpus(workloads.C3_SMALL)
    fds = np.array([os.open(p, os.O_RDONLY) for p in corpus.paths], np.int32)
    sizes = np.array([os.path.getsize(p) for p in corpus.paths], np.uint64)
    q, ql = _pack_queries(corpus.queries)
    nq = len(corpus.queries)
    chunk, ctas, threads = 16 << 10, 148, 256
    with G.Context(device=0, service_threads=4, staging_bytes=64 << 20) as ctx:
        need = ctas * (chunk + 64) * 2
        st = ctx.staging(need)
        try:
            ref = torch.zeros(nq, dtype=torch.int64, device="cuda")
            rc = L.genesys_c3_wordcount(ctx.handle, fds.ctypes.data, sizes.ctypes.data, len(fds), q.ctypes.data,
                                        ql.ctypes.data, nq, chunk, ctas, threads, G.FORM_BATCHED, st, need,
                                        ref.data_ptr(), None)
            assert rc == 0, G.last_error()
            want = ref.cpu().numpy()
            assert want.sum() > 0
            assert np.array_equal(want.astype(np.uint64), corpus.truth_total())
            device_before = torch.cuda.current_device()
            for call in range(2):
                got = torch.zeros(nq, dtype=torch.int64, device="cuda")
                rc = L.genesys_c3_wordcount_noalloc(ctx.handle, fds.ctypes.data, sizes.ctypes.data, len(fds),
                                                    q.ctypes.data, ql.ctypes.data, nq, chunk, ctas, threads,
                                                    G.FORM_BATCHED, st, need, got.data_ptr(), None)
                assert rc == 0, (call, G.last_error())
                assert torch.cuda.current_device() == device_before, call
                assert np.array_equal(got.cpu().numpy(), want), call
                assert np.array_equal(got.cpu().numpy().astype(np.uint64), corpus.truth_total()), call
            # inputs needing more work items than the fixed array holds are refused
            too_small_chunk = 64
            n_items = int(sum(-(-int(s) // too_small_chunk) for s in sizes))
            assert n_items > 32768
            rc = L.genesys_c3_wordcount_noalloc(ctx.handle, fds.ctypes.data, sizes.ctypes.data, len(fds),
                                                q.ctypes.data, ql.ctypes.data, nq, too_small_chunk, ctas, threads,
                                                G.FORM_BATCHED, st, need, got.data_ptr(), None)
            assert rc == G.EINVAL
            assert "at most 32768" in G.last_error()
        finally:
            for fd in fds:
                os.close(int(fd))
