"""Run by tests/test_gpu_checked.py in a child process with
GENESYS_LIBRARY=checked: the device-side index checks are compiled in, and a
few workloads must give the oracle's results with every status word zero."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
import paper_1705_06965_b300 as G  # noqa: E402
import workloads  # noqa: E402


def main(tmp: str) -> None:
    assert G.LIB_PATH.endswith("libgenesys_checked.so"), G.LIB_PATH
    torch.cuda.set_device(0)
    with G.Context(device=0, service_threads=4, staging_bytes=64 << 20, deadline_ns=5_000_000_000) as ctx:
        # C1, every form
        p = workloads.c1_file(os.path.join(tmp, "c1.bin"), (1 << 20) + 77, seed=11)
        want = oracle.c1_histogram(p, 4096)
        st = ctx.staging(16 << 20)
        for form in (G.FORM_PLAIN, G.FORM_BATCHED, G.FORM_WARP, G.FORM_HBM):
            h = torch.zeros(256, dtype=torch.int32, device="cuda")
            fd = os.open(p, os.O_RDONLY)
            ctx.c1_histogram(fd, os.path.getsize(p), h.data_ptr(), st, 16 << 20, chunk=4096, groups=32, threads=256,
                             form=form)
            os.close(fd)
            assert np.array_equal(h.cpu().numpy().view(np.uint32), want), form
        # C2, every grain
        n = 4096 + 37
        for gran, bt in ((0, 256), (1, 256), (2, 128), (3, 256)):
            q = os.path.join(tmp, f"c2_{gran}.bin")
            fd = os.open(q, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
            ctx.c2_pwrite(fd, n, gran, bt, gran != 0, False, workloads.SEED_C2, st, n * 64)
            os.close(fd)
            w = os.path.join(tmp, f"w_{gran}.bin")
            oracle.c2_pwrite(w, n, {0: 1, 1: 32, 2: bt, 3: n}[gran])
            assert open(q, "rb").read() == open(w, "rb").read(), gran
        # C3, the small corpus
        c = workloads.corpus(workloads.C3_SMALL)
        fds = [os.open(x, os.O_RDONLY) for x in c.paths]
        counts = torch.zeros(len(c.queries), dtype=torch.int64, device="cuda")
        ctx.staging_reset()
        sb = 2 * 64 * ((64 << 10) + 64)
        st = ctx.staging(sb)
        ctx.c3_wordcount(fds, c.sizes, c.queries, counts.data_ptr(), st, sb, chunk=64 << 10, ctas=64, threads=512,
                         form=G.FORM_BATCHED)
        for fd in fds:
            os.close(fd)
        assert np.array_equal(counts.cpu().numpy().astype(np.uint64), c.truth_total())
        assert ctx.status() == [0] * G.ST_WORDS, ctx.status()
        assert ctx.stats()["protocol_errors"] == 0
    short_reads(tmp)
    print("checked ok")


def short_reads(tmp: str, cap: int = 1000) -> None:
    """Every pread the service threads make asks for at most `cap` bytes, so
    the GPU's readers meet short reads in the middle of files (merged calls
    included): C1 in every form, C3 in both forms and C5's preads must go on
    reading and still give the oracle's results."""
    with G.Context(device=0, service_threads=4, staging_bytes=64 << 20, deadline_ns=5_000_000_000) as ctx:
        ctx.pread_cap(cap)
        p = workloads.c1_file(os.path.join(tmp, "c1s.bin"), (1 << 20) + 77, seed=12)
        want = oracle.c1_histogram(p, 4096)
        st = ctx.staging(16 << 20)
        before = ctx.stats()
        for form in (G.FORM_PLAIN, G.FORM_BATCHED, G.FORM_WARP, G.FORM_HBM):
            h = torch.zeros(256, dtype=torch.int32, device="cuda")
            fd = os.open(p, os.O_RDONLY)
            ctx.c1_histogram(fd, os.path.getsize(p), h.data_ptr(), st, 16 << 20, chunk=4096, groups=32, threads=256,
                             form=form)
            os.close(fd)
            assert np.array_equal(h.cpu().numpy().view(np.uint32), want), ("short reads", form)
        after = ctx.stats()
        # 4 forms x ceil((1 MiB + 77) / 1000) capped reads at least: the cap was in force
        assert after["by_op"]["pread"] - before["by_op"]["pread"] >= 4 * ((1 << 20) + 77) // cap
        c = workloads.corpus(workloads.C3_SMALL)
        fds = [os.open(x, os.O_RDONLY) for x in c.paths]
        ctx.staging_reset()
        sb = 2 * 64 * ((64 << 10) + 64)
        st = ctx.staging(sb)
        for form in (G.FORM_PLAIN, G.FORM_BATCHED):
            counts = torch.zeros(len(c.queries), dtype=torch.int64, device="cuda")
            ctx.c3_wordcount(fds, c.sizes, c.queries, counts.data_ptr(), st, sb, chunk=64 << 10, ctas=64,
                             threads=512, form=form)
            assert np.array_equal(counts.cpu().numpy().astype(np.uint64), c.truth_total()), ("short reads", form)
        for fd in fds:
            os.close(fd)
        ctx.staging_reset()
        tr = workloads.c5_trace(workloads.C5_SMALL).subset(np.arange(40))
        out = os.path.join(tmp, "c5s.bin")
        ref = os.path.join(tmp, "c5s_ref.bin")
        in_fds = [os.open(x, os.O_RDONLY) for x in tr.in_paths]
        ofd = os.open(out, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        rfd = os.open(ref, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        try:
            res, _, _ = ctx.c5_serve(tr.arrival_ns, tr.threads, tr.n_ops, tr.ops, in_fds, ofd, max_inflight=8,
                                     honor_arrivals=0, staging_budget=32 << 20)
            want5 = oracle.c5_trace(tr, rfd, in_fds)
        finally:
            for fd in in_fds + [ofd, rfd]:
                os.close(fd)
        m = np.arange(8)[None, :] < tr.n_ops[:, None]
        assert np.array_equal(res[m], want5[m]), "short reads: C5 results"
        assert open(out, "rb").read() == open(ref, "rb").read(), "short reads: C5 output file"
        assert ctx.status() == [0] * G.ST_WORDS, ctx.status()


if __name__ == "__main__":
    main(sys.argv[1])
