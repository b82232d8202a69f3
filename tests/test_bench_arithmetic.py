"""The benchmark's own arithmetic, pinned on the CPU: the syscall count that
is the headline's numerator equals the calls the oracle issues for the same
sweep, and the clock record that decides whether a run is rejected is read
correctly."""
import os

import pytest

import bench
import oracle
import workloads


@pytest.mark.parametrize("n", [1000, 4096])
def test_calls_per_combination_equal_the_oracles_issued_calls(tmp_path, n):
    """One call per work-item, per warp of 32, per work-group, per kernel:
    what calls_for counts is what the oracle issues when it groups the same
    threads that way (ragged last groups included)."""
    p = str(tmp_path / "c2.bin")
    for name, g, bt, relaxed, nb in bench.COMBOS:
        group = {0: 1, 1: 32, 2: bt, 3: n}[g]
        assert bench.calls_for(g, bt, n) == oracle.c2_pwrite(p, n, group, bench.SEED_C2), (name, relaxed, nb)


def test_step_call_count_equals_the_reference_arms():
    """The GPU arm's syscalls per step (step_calls) and the reference arm's
    (oracle_step, the whole sweep plus the C1 preads) are the same number."""
    c2, c1 = bench.step_calls()
    calls, _, full = bench.oracle_step(workloads.scratch_dir("test_bench_arith"))
    assert full and calls == c2 + c1
    assert c1 == 2 * (bench.C1_BYTES // bench.C1_CHUNK)


def test_clock_record_reasons_and_median(tmp_path):
    """nvidia-smi's CSV as the sampler writes it: the median SM clock, the
    maximum, and every throttle reason seen active at least once."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.p = object()  # as if the sampler had run
    head = ("index, clocks.current.sm [MHz], clocks.max.sm [MHz], power.draw [W], clocks_event_reasons.active, "
            "clocks_event_reasons.hw_slowdown, clocks_event_reasons.hw_thermal_slowdown, "
            "clocks_event_reasons.sw_thermal_slowdown, clocks_event_reasons.sw_power_cap")
    rows = ["0, 2032 MHz, 2032 MHz, 700.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980 MHz, 2032 MHz, 1090.00 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2010 MHz, 2032 MHz, 900.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    open(s.path, "w").write("\n".join([head] + rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2032.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    open(s.path, "w").write("\n".join([head, rows[0].replace("Not Active, Not Active, Not Active, Not Active",
                                                              "Active, Not Active, Not Active, Not Active")]) + "\n")
    assert bench.ClockSampler.summary(s)["reasons"] == ["hw_slowdown"]
    s.p = None
    assert bench.ClockSampler.summary(s)["sm_mhz"] is None


def test_traffic_figure_is_scaled_and_dropped_when_the_source_changes(tmp_path, monkeypatch):
    """The roofline's traffic: the committed per-thread figure times the
    threads of a launch, and no figure at all once the kernel's source (the
    device protocol headers or its section of workloads.cu) differs from the
    one the capture was taken on."""
    import shutil
    root = bench.ROOT
    for rel in ("include/genesys_device.cuh", "include/genesys_layout.h",
                "paper_1705_06965_b300/csrc/workloads.cu"):
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(root, rel), tmp_path / rel)
    kern = "c2_pwrite_kernel<work-item,strong,blocking>"
    h = bench.kernel_src_hash(kern)
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "traffic.txt").write_text(f"# comment\n{kern} {h} 243.5 thread x\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_src_hash(kern) == h
    assert bench.load_traffic(kern, 1 << 20) == round(243.5 * (1 << 20))
    assert bench.load_traffic("c2_pwrite_kernel<warp,strong,blocking>", 1 << 20) is None
    with open(tmp_path / "include" / "genesys_device.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.kernel_src_hash(kern) != h
    assert bench.load_traffic(kern, 1 << 20) is None


def test_cpu_baseline_leg_compares_the_gpu_histogram_with_the_oracle():
    """The GPU arm hands its C1 histogram to the CPU-baseline leg, which
    reports whether it equals the oracle's for the same seeded file; the
    arm's own check (forms agree, every byte counted) holds for the oracle's
    histogram too."""
    import numpy as np
    want = oracle.c1_histogram(workloads.c1_file(None, bench.C1_BYTES, seed=workloads.SEED_C1), bench.C1_CHUNK)
    assert int(want.sum(dtype=np.uint64)) == bench.C1_BYTES
    out = bench.cpu_baseline_sample(budget_s=0.5, c1_hist=want.copy())
    assert out["kind"] == "oracle" and out["c1_histogram_equals_oracle"] is True
    bad = want.copy()
    bad[7] += 1
    assert bench.cpu_baseline_sample(budget_s=0.5, c1_hist=bad)["c1_histogram_equals_oracle"] is False


def _full_line():
    """A bench line with every section the summary reads, at realistic sizes."""
    pt = lambda rate, got, late: {"requests": 1000, "received": got, "served": got,  # noqa: E731
                                   "achieved_req_per_s": rate, "p50_us": 41.234567, "p99_us": 812.98765,
                                   "max_send_late_us": 12.3, "offered_on_schedule": late}
    return {
        "value": 9752850.612345, "e2e": {"value": 9727511.123},
        "forms": {"plain_blocking_strong": {"syscalls_per_s": 31600000.1, "requests_per_s": 31600000.1,
                                            "p50_us": 300.1, "p99_us": 900.2},
                  "batched": {"syscalls_per_s": 84000.5, "requests_per_s": 86000000.3, "p50_us": 200.1,
                              "p99_us": 700.7},
                  "plain_per_call_service": {"syscalls_per_s": 9000000.2, "requests_per_s": 9000000.2,
                                             "p50_us": 9000.1, "p99_us": 20000.2}},
        "roofline": {"service": {"achieved": 33400000.2, "frac": 0.181234,
                                 "warp_interleaved_order": {"frac": 0.347712}}},
        "c1_4MiB": {"plain": {"GB_per_s": 5.31123, "preads_per_s": 1296000.3, "p99_us": 612.34},
                    "batched": {"GB_per_s": 7.7789, "preads_per_s": 1899000.1, "p99_us": 701.2}},
        "pread_scan_1GiB": {"autotuned": {"form": 0}, "plain": {"GB_per_s": 49.712, "frac_of_host_link_h2d": 0.894},
                            "warp": {"GB_per_s": 51.1, "frac_of_host_link_h2d": 0.919,
                                     "frac_of_sm_zero_copy_read": 0.98765},
                            "batched": {"GB_per_s": 47.2, "frac_of_host_link_h2d": 0.849}},
        "wordcount_c3": {"plain": {"GB_per_s": 40.1, "frac_of_host_link_h2d": 0.72, "counts_equal_ground_truth": True},
                         "batched": {"GB_per_s": 49.5, "frac_of_host_link_h2d": 0.89,
                                     "counts_equal_ground_truth": True},
                         "cpu_baseline_oracle": {"one_thread_GB_per_s": 0.131, "files_to_cores_GB_per_s": 0.771}},
        "kv_c4": {"rates": {"50000": pt(49999.9, 1000, True), "800000": pt(799012.3, 1000, True),
                            "1600000": pt(1300123.4, 1000, False)},
                  "saturation_req_per_s": 799012.3, "saturation_p50_us": 41.234567, "saturation_p99_us": 812.98765,
                  "best_any_req_per_s": 1300123.4, "saturation_host_bound": True,
                  "cpu_baseline_oracle_server": {"saturation_req_per_s": 270123.1}},
        "served_c5": {"plain_first1000": {"requests_per_s": 2100.3, "syscalls_per_s": 57000.1, "p99_ms": 447.12},
                      "served_first1000": {"requests_per_s": 8800.2, "syscalls_per_s": 240000.7, "p99_ms": 65.3},
                      "persistent_first1000": {"requests_per_s": 12000.2, "syscalls_per_s": 330000.7, "p99_ms": 30.3},
                      "served_full": {"requests_per_s": 8700.1, "p99_ms": 70.123},
                      "persistent_full": {"requests_per_s": 11000.1, "p99_ms": 40.123,
                                          "link": {"frac_h2d": 0.63456, "frac_d2h": 0.59123,
                                                   "frac_sm_both": 0.90111}},
                      "first1000_alone_equals_mix": True,
                      "cpu_baseline_oracle_replay_first1000": {"requests_per_s": 174.2}},
        "probes": {"host_cpus": 16},
        "cpu_baseline": {"value": 1293220.2, "c1_histogram_equals_oracle": True},
        "oracle_checks": {"ran": True, "c4_replies_equal": True, "c5_full_equal": True},
    }


def test_summary_fits_the_kept_tail_and_carries_every_config():
    """The driver keeps the last 1,500 characters of the bench line: the
    summary (the line's last key, targets inside) must fit with room to spare
    and hold a figure for every config."""
    import json
    line = _full_line()
    line["summary"] = bench.summarize(line)
    tail = json.dumps(line)[-1500:]
    assert '"summary": {' in tail and '"targets": {' in tail
    sm = line["summary"]
    assert len(json.dumps(sm)) <= 1350, len(json.dumps(sm))
    assert sm["scan_1GiB"] == {"form": "warp", "GBps": 51.1, "frac_h2d": 0.919, "frac_sm_read": 0.988}
    assert sm["wi_2p20"] == {"calls_per_s": 33400000, "frac_file_order": 0.181, "frac_interleaved": 0.348}
    assert sm["c3"]["GBps"] == 49.5 and sm["c3"]["truth_eq"] is True
    assert sm["c4"]["sat_rps"] == 799000 and sm["c4"]["replies_eq_oracle"] is True
    assert sm["c4"]["p99_us"] == 813 and sm["c4"]["best_any_rps"] == 1300000
    assert sm["c5"]["persistent_rps"] == 11000 and sm["c5"]["full_eq_oracle"] is True
    assert sm["c5"]["persistent_link_frac"] == [0.635, 0.591, 0.901]
    assert sm["oracle"]["cores"] == 16 and sm["oracle"]["c5_rps_1t"] == 174
    t = sm["targets"]
    assert t["c2_batched_beats_plain"] == {"syscalls_per_s": True, "p99": True}
    assert t["c2_coarse_grain_beats_work_item"] == {"syscalls_per_s": False, "requests_per_s": True, "p99": True}
    assert t["c1_batched_beats_plain"] == {"syscalls_per_s": True, "p99": False}
    assert t["c5_served_beats_plain"] == {"syscalls_per_s": True, "requests_per_s": True, "p99": True}
    assert t["pread_scan_frac_h2d_ge_0.75"] == {"scan_1GiB": True, "c3": True}
    assert t["c3_batched_beats_plain"] is True


def test_summary_of_a_line_without_extras():
    """--extras 0 lines (launch lists) still get a summary, with None where a
    section was not measured."""
    sm = bench.summarize({"value": 1.0, "e2e": {"value": 1.0}})
    assert sm["c4"]["sat_rps"] is None and sm["targets"]["pread_scan_frac_h2d_ge_0.75"]["scan_1GiB"] is None
    assert sm["targets"]["c5_served_beats_plain"]["p99"] is None


def test_kv_saturation_counts_only_points_offered_on_schedule():
    """A point where the load generator fell behind its own schedule measures
    the host: the saturation point is the best clean point, and the sweep is
    marked host-bound when it ended on such a point."""
    pts = _full_line()["kv_c4"]["rates"]
    sat = bench.kv_saturation(pts)
    assert sat["saturation_req_per_s"] == 799012.3 and sat["best_any_req_per_s"] == 1300123.4
    assert sat["saturation_host_bound"] is True
    pts["800000"]["received"] = 999                  # a reply missing: not a clean point either
    assert bench.kv_saturation(pts)["saturation_req_per_s"] == 49999.9
    assert bench.kv_saturation({})["saturation_req_per_s"] is None


def test_reply_digests_tell_replies_apart():
    import numpy as np
    d = bench.reply_digests([b"", b"\x80\x00\x10\x00abcd", b"\x80\x00\x10\x00abce", b"\x81\x00\x00\x00" + b"\0" * 4])
    assert d.dtype == np.uint64 and len(set(d.tolist())) == 4 and d[0] == 0


def test_c5_link_bytes_counts_each_direction():
    """pread bytes come in, pwrite bytes go out, an mmap'd region goes out
    (the fill) and comes back (the checksum's read); operations past a
    request's count are not counted."""
    import numpy as np
    import workloads
    ops = np.zeros((2, workloads.C5_MAX_OPS), workloads.C5_OP)
    ops[0, 0] = (workloads.OP_PREAD, 0, 0, 1000, 0, 0)
    ops[0, 1] = (workloads.OP_MMAP, 0, 0, 8192, 0, 0)
    ops[0, 2] = (workloads.OP_PWRITE, 0, 0, 999999, 0, 0)       # past n_ops: not run
    ops[1, 0] = (workloads.OP_PWRITE, 0, 0, 300, 0, 0)
    tr = workloads.Trace(np.zeros(2, np.uint64), np.array([64, 64], np.uint32), np.array([2, 1], np.uint32), ops,
                         [], 300)
    assert bench.c5_link_bytes(tr) == (1000 + 8192, 300 + 8192)
