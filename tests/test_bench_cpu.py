"""CPU checks of bench.py's measurement helpers: the roofline arithmetic (algorithmic bytes per launch
over the push's event time), the rule that the profiled DRAM traffic is reported only for the kernel
source it was captured on, the clock-sample parsing, and the oracle timing over several host threads."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_arithmetic():
    # 16.8M particles at 48 B (cell index, offsets, momenta each way) and 0.5M cells at 36 B, 10
    # launches in 5 ms: 0.5 ms per launch; the layout's own 40 B per particle beside it
    np_, ncell = 16777216, 524288
    rf = bench.roofline({"push": (5.0, 10)}, np_, ncell, 4, 6791.4, "measured")
    want_bytes = np_ * 48 + ncell * 36
    assert rf["algorithmic_bytes_per_launch"] == want_bytes
    assert abs(rf["achieved"] - want_bytes / 0.5e-3 / 1e9) < 0.1
    assert abs(rf["frac"] - rf["achieved"] / 6791.4) < 1e-4
    assert rf["launch_ms"] == 0.5 and rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert abs(rf["frac_layout_bytes"] - (np_ * 40 + ncell * 36) / 0.5e-3 / 1e9 / 6791.4) < 1e-4
    assert rf["time_basis"] == "event-bracketed launches"


def test_push_time_from_the_graph_replayed_step():
    # step of 0.6 ms in the graph; the timed pass of 10 single steps: push 5 ms, the rest 1 ms in all,
    # so the push takes 0.6 - 0.1 = 0.5 ms of a replayed step
    kt = {"push": (5.0, 10), "copies": (0.4, 10), "yee": (0.5, 10), "migrate": (0.1, 10)}
    assert abs(bench.push_time_in_step(kt, 0.6) - 0.5) < 1e-12
    rf = bench.roofline(kt, 16777216, 524288, 4, 6791.4, "measured", step_ms=0.6)
    assert rf["launch_ms"] == 0.5 and rf["launch_ms_events"] == 0.5
    assert rf["time_basis"].startswith("graph-replayed")
    assert bench.push_time_in_step(kt, 0.05) is None  # less than the other kernels: no estimate


def test_median_kernel_times_ignores_one_stray_launch():
    # five steps; one of them caught a slow spill launch: the median per class is unmoved
    steps = [{"push": (0.33, 1), "spill": (0.006, 1)} for _ in range(5)]
    steps[2] = {"push": (0.33, 1), "spill": (0.089, 1)}
    kt = bench.median_kernel_times(steps)
    assert abs(kt["spill"][0] / 5 - 0.006) < 1e-12 and kt["spill"][1] == 5
    assert abs(kt["push"][0] - 5 * 0.33) < 1e-12
    even = bench.median_kernel_times(steps[:4])
    assert abs(even["spill"][0] / 4 - 0.006) < 1e-12


def test_warm_up_runs_one_call_long_enough_to_capture_the_graph():
    # the warm-up is one pic_step call of at least 4 steps (two graphs' worth at one step per
    # energy record), so the step graph is captured before the timed call replays it
    calls = []

    class FakeP:
        @staticmethod
        def pic_step(h, n):
            calls.append((h, n))

    bench.warm_up(FakeP, "h", 3)
    bench.warm_up(FakeP, "h", 7)
    assert calls == [("h", 4), ("h", 7)]


def test_bin_stats_reports_capacity_and_spills():
    class FakeP:
        @staticmethod
        def pic_bin_stats(h):
            return 48, 12

    assert bench.bin_stats(FakeP, None) == {"capacity": 48, "spilled": 12}


def test_traffic_only_for_the_profiled_source(tmp_path):
    src = tmp_path / "kernel.cu"
    src.write_text("kernel source\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profile.md"
    prof.write_text(f"# summary\n\nsource_sha256: {digest}\ndram_bytes_per_launch: 123456\n")
    assert bench.profiled_traffic(str(prof), str(src)) == 123456.0
    src.write_text("kernel source, changed\n")
    assert bench.profiled_traffic(str(prof), str(src)) is None
    assert bench.profiled_traffic(str(tmp_path / "missing.md"), str(src)) is None
    # several files: one digest over their bytes in order; a change in any of them drops the figure
    hdr = tmp_path / "tile.cuh"
    hdr.write_text("tile shape\n")
    both = hashlib.sha256(src.read_bytes() + hdr.read_bytes()).hexdigest()
    prof.write_text(f"source_sha256: {both}\ndram_bytes_per_launch: 42\n")
    assert bench.profiled_traffic(str(prof), [str(src), str(hdr)]) == 42.0
    hdr.write_text("tile shape, changed\n")
    assert bench.profiled_traffic(str(prof), [str(src), str(hdr)]) is None


def test_clock_sample_parsing():
    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ])
    c = bench.parse_clock_samples(text)
    assert c["samples"] == 3 and c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    hot = bench.parse_clock_samples("0, 1500, 2070, 1400, 0x20, Not Active, Active, Not Active, Not Active")
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.parse_clock_samples("")["sm_mhz"] is None


def test_oracle_timing_over_threads():
    # two concurrent slabs (seeds 2 and 3) of a thin 512 x 8 sample: the particle count is both slabs',
    # one wall time per timed step, and the slabs are distinct samples of the same beam
    n1, t1 = bench.oracle_time(1, 0, nz=8, threads=1)
    n2, t2 = bench.oracle_time(2, 1, nz=8, threads=2)
    assert n1 == bench.NX * 8 * 2 * bench.PPC and n2 == 2 * n1
    assert len(t1) == 1 and len(t2) == 2 and min(t2) > 0
    a, b = bench.oracle_sample(8, seed=2), bench.oracle_sample(8, seed=3)
    assert a.n == b.n and not (a.part["z"] == b.part["z"]).all()


def test_cgroup_cpu_limit_parsing():
    assert bench.cgroup_cpu_limit("max 100000\n") is None
    assert bench.cgroup_cpu_limit("1600000 100000\n") == 16
    assert bench.cgroup_cpu_limit("150000 100000") == 1
    assert bench.cgroup_cpu_limit("50000 100000") == 1
    assert bench.cgroup_cpu_limit("") is None and bench.cgroup_cpu_limit("x y") is None
    assert 1 <= bench.host_threads() <= (os.cpu_count() or 1)


def test_oracle_baseline_of_the_3d_workload():
    # two concurrent 128 x 128 x 2 slabs of the 3D workload, one step each: the count is both slabs'
    # particles (8 per cell and species) and the line carries the baseline's keys
    cb = bench.cpu_baseline_3d(steps=1, threads=2, nz=2)
    assert cb["cores"] == 2 and cb["kind"] == "oracle" and cb["value"] > 0
    assert "128x128x2" in cb["sample"] and f"{128 * 128 * 2 * 16} particles a slab" in cb["sample"]


def test_oracle_baseline_of_the_small_workload():
    cb = bench.oracle_config1(steps=2)
    assert cb["cores"] == 1 and cb["kind"] == "oracle" and cb["value"] > 0
    assert "65536 particles" in cb["sample"]
