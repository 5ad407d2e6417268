"""The benchmark's roofline arithmetic on the CPU: the algorithmic operation
counts per walk-step that the bench divides by, the peaks it derives from the
SM count and clock, and the fraction it reports (no GPU, no oracle)."""
import math

import pytest

import bench as B


def test_counts_per_walk_step():
    # torus, one Philox block per step (the table in bench.py's comment sums to 148)
    assert B.OPS_PER_STEP == 148
    # full sampler at n = 1000: 62.5 groups x (Z 218 + Theta 242) + 200 scalar
    assert B.ops_full_sampler(1000) == pytest.approx(62.5 * (218 + 242) + 200)
    assert B.ops_full_sampler(1000) == pytest.approx(28_950)
    # Example 2 (n = 1001): Z adds the revolution's v and A terms
    assert round(B.ops_full_sampler(1001, revolution=True)) == 33_859
    # tensor-core walk at n = 1000: 2 n components, 15.625 per component + 300
    assert B.ops_tc_embedded(1000) == pytest.approx(2000 * (198 / 16 + 3.25) + 300)
    assert B.ops_tc_embedded(1000) == pytest.approx(31_550)
    # reduced sampler: S^999 (two directions of 132.25 + 80) and S^20 (D = 21)
    assert B.OPS_REDUCED_S999 == pytest.approx(344.5)
    D = 21
    direction = 40 * math.ceil(D / 4) + 11.75 * math.ceil(D / 2) + 68.75
    assert B.ops_reduced_embedded(20) == pytest.approx(2 * direction + 2 * (3 * D + 2) + D * D + 2 * D + 80)
    assert B.ops_reduced_embedded(20) == pytest.approx(1_569)


def test_peaks_from_sm_count_and_clock():
    assert B.issue_peak(148, 2032.0) == pytest.approx(148 * 4 * 32 * 2.032e9)
    assert B.mufu_peak(148, 2032.0) == pytest.approx(148 * 16 * 2.032e9)
    assert B.issue_peak(148, 2032.0) / B.mufu_peak(148, 2032.0) == pytest.approx(8.0)


def test_roofline_fraction():
    # 2.1504e10 walk-steps (4096 x 1e4 x 525) in 136.4 ms at 148 ops per step
    rb = B.roofline_block("k", B.OPS_PER_STEP, 2.1504e10, 0.1364, 148, 2032.0, "measured",
                          mufu_per_step=4000)
    achieved = 148 * 2.1504e10 / 0.1364
    assert rb["frac"] == pytest.approx(achieved / (148 * 4 * 32 * 2.032e9))
    assert 0.6 < rb["frac"] < 0.62
    assert rb["achieved"] == pytest.approx(achieved / 1e12)
    assert rb["mufu"]["frac"] == pytest.approx(4000 * 2.1504e10 / 0.1364 / (148 * 16 * 2.032e9))


def test_traffic_is_the_captured_dram_bytes():
    # read + write of one bench launch (ncu), within the 655 MB of per-walk outputs
    assert 600e6 < B.TRAFFIC_BYTES < 655e6
