"""Host-side pieces of the benchmark (no GPU): the clock record's parsing and the reading of the
committed ncu summary."""
import bench
from paper_2103_14294_b300.clocks import ClockSampler


def test_clock_summary_median_under_load_and_reasons():
    c = ClockSampler(0)
    c.lines = [
        "2032, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1980, 2032, 1090.5, 0x4, Not Active, Not Active, Not Active, Active",
        "345, 2032, 120.0, 0x1, Not Active, Not Active, Not Active, Not Active",  # idle: not "under load"
        "garbage line",
        "[N/A], 2032, 100, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2032.0
    assert s["sm_mhz"] == 2006.0  # median of the two samples above 30% of the maximum
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_samples():
    assert ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_committed_ncu_summary_matches_the_kernel_source():
    """The bench quotes DRAM bytes per algorithmic byte from the committed ncu summary only while
    that summary's kernel hash equals the current kernel source's."""
    prof = bench.ncu_profile()
    assert set(prof) >= {"k4", "c4"}
    for q in ("k4", "c4"):
        assert 0 < prof[q]["dram_bytes_per_alg_byte"] < 1
        assert 0 < prof[q]["l2_hit_pct"] <= 100


def test_single_rank_totals_are_the_local_ones():
    assert bench.job_totals(1.5, 10, None, 1) == (1.5, 10.0)
