"""Host-side logic of bench.py (no GPU): the roofline's algorithmic bytes,
the measured peak, the profiled DRAM traffic gated on the kernel source's
hash, and the clock-sample summary that decides whether a run is rejected."""
import hashlib
import importlib.util
import os

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(REPO, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_of_the_pagerank_superstep(bench):
    # 8 B per edge + 16 B per vertex: 604.0 MB at R-MAT 22 (20 B per vertex, 620.8 MB,
    # with the old-rank read of the L1 delta)
    assert bench.algorithmic_bytes(1 << 22, 1 << 26) == 8 * (1 << 26) + 16 * (1 << 22) == 603979776
    assert bench.algorithmic_bytes_with_old_rank(1 << 22, 1 << 26) == 620756992


def test_measured_peak_is_the_driver_file(bench):
    p = bench.measured_peaks()
    assert p["source"] == "measured" and p["hbm_gbs"] > 1000


def test_traffic_only_while_the_profile_matches_the_kernel(bench, tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    prof = tmp_path / "profile.txt"
    prof.write_text(f"# comment: ignored\nkernel_source_sha256: {sha}\ndram_bytes_per_launch: 12345\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profiled_traffic() == 12345.0
    assert bench.profiled_traffic(str(prof)) == 12345.0
    src.write_text("kernel v2")          # the kernel changed since the counters were taken
    assert bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.txt"))
    assert bench.profiled_traffic() is None


def test_committed_profile_matches_the_committed_kernel(bench):
    # the PageRank summary under profiles/ was taken on the kernel as committed
    assert bench.profiled_traffic() is not None


def test_clock_summary_flags_throttling(bench):
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2070.0 and s["sm_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    empty = bench.ClockSampler(0)
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_cc_roofline_averages_the_full_sweeps(bench):
    # the last superstep pushed (a few out-edges): it is not a sweep of every edge
    us, n = bench.sweep_launch_us([1.2, 1.0, 0.1], [True, True, False])
    assert n == 2 and abs(us - 1100.0) < 1e-9
    us, n = bench.sweep_launch_us([0.2, 0.4], [False, False])
    assert n == 2 and abs(us - 300.0) < 1e-9
