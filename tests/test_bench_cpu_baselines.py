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
