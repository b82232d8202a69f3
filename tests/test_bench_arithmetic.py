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
