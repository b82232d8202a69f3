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


def test_oracle_checks_of_the_c2_files_and_the_scan(tmp_path):
    """The bench's oracle leg compares the files the sweep wrote and the scan's
    histogram with the oracle's, and a one-byte difference in either shows."""
    import numpy as np
    import oracle
    import workloads
    n = 1000
    c2 = tmp_path / "c2.bin"
    want = tmp_path / "want.bin"
    oracle.c2_pwrite(str(want), n, 32, bench.SEED_C2)      # written another way: a warp's calls
    c2.write_bytes(want.read_bytes())
    scan = workloads.c1_file(str(tmp_path / "scan.bin"), 100_000, seed=7)
    hist = oracle.c1_histogram(scan, 4096)
    out = bench.oracle_checks({"c2_files": [(n, str(c2))], "scan": (scan, hist.copy())})
    assert out["c2_files_equal"] is True and out["scan_1GiB_histogram_equal"] is True
    data = bytearray(c2.read_bytes())
    data[12345] ^= 1
    c2.write_bytes(bytes(data))
    bad = hist.copy()
    bad[3] += 1
    bad[4] -= 1
    out = bench.oracle_checks({"c2_files": [(n, str(c2))], "scan": (scan, bad)})
    assert out["c2_files_equal"] is False and out["scan_1GiB_histogram_equal"] is False
    assert not (tmp_path / "c2.bin.oracle").exists()
