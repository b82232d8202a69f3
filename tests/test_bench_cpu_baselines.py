"""The benchmark's CPU baselines for C3 and C5 (the oracle timed on the host
cores): on the small configurations, the numbers are filled in, the
one-thread and files-to-cores wordcounts agree, and the replay's agreement
check notices a result that differs."""
import os

import numpy as np

import bench
import oracle
import workloads


def test_c3_baseline_counts_agree_across_forms():
    c = workloads.corpus(workloads.C3_SMALL)
    r = bench.cpu_baseline_c3(c, sample_bytes=256 << 10)
    assert r["kind"] == "oracle" and r["counts_agree"]
    assert r["one_thread_GB_per_s"] > 0 and r["files_to_cores_GB_per_s"] > 0 and r["cores"] >= 1
    assert r["sample"].startswith("first ")


def test_c5_baseline_replay_checks_the_served_results():
    tr = workloads.c5_trace(workloads.C5_SMALL)
    sub = tr.subset(np.arange(50))
    d = workloads.scratch_dir("test_bench_c5_baseline")
    in_fds = [os.open(p, os.O_RDONLY) for p in tr.in_paths]
    try:
        ofd = os.open(os.path.join(d, "ref.bin"), os.O_CREAT | os.O_RDWR, 0o644)
        try:
            ref = oracle.c5_trace(sub, ofd, in_fds)
        finally:
            os.close(ofd)
        r = bench.cpu_baseline_c5(sub, in_fds, d, ref)
        assert r["served_results_equal_oracle"] and r["requests"] == 50 and r["requests_per_s"] > 0
        bad = ref.copy()
        bad[7, 0] ^= 1
        assert not bench.cpu_baseline_c5(sub, in_fds, d, bad)["served_results_equal_oracle"]
    finally:
        for fd in in_fds:
            os.close(fd)


def test_service_phases_from_a_host_only_context(tmp_path):
    """The per-request service breakdown the bench reports: with emulated
    callers on a host-only context every phase is filled in, and ordering,
    Linux calls and completion together fit in the batch-processing time."""
    import paper_1705_06965_b300 as G
    n = 4096
    fd = os.open(str(tmp_path / "p.bin"), os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o600)
    try:
        with G.Context(host_only=True, service_threads=2, coalesce_max=256, staging_bytes=n * 64 + 4096) as c:
            buf = c.staging(n * 64)
            before = c.stats()
            assert c.service_probe(fd, buf, 64, n) > 0
            ph = bench.service_phases(before, c.stats())
    finally:
        os.close(fd)
    assert set(ph) == {"pickup", "order", "os_call", "complete", "busy", "requests_per_batch", "requests_per_os_call",
                       "empty_polls_per_batch", "hole_polls_per_batch"}
    assert all(v >= 0 for v in ph.values()) and ph["os_call"] > 0 and ph["requests_per_batch"] >= 1
    assert ph["order"] + ph["os_call"] <= ph["busy"] + 1e-6
