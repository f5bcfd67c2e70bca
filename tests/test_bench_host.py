"""Host-side pieces of bench.py (no GPU): the committed ncu summaries it reads its
roofline basis from parse, and the basis is the issue budget over their count."""
import math

import bench


def test_profile_summaries_are_current_and_parse():
    for path in (bench.PROFILE_SUMMARY, bench.GAUSS_PROFILE_SUMMARY):
        ops, per_clk, kind, _ = bench.ops_per_update(path)
        assert ops and ops > 1.0 and per_clk == 64.0 and kind, path
    # traffic is read only from a summary taken on the current source and launch shapes
    t = bench.profile_traffic(tail=bench.tail_kernel(10, {"words": 16, "threads": 320, "ctas_per_sm": 2}))
    assert t is None or t > 1e9
    assert bench.profile_traffic(kernel="k_sweep<10,8,160,3>") is None


def test_issue_peak_is_the_issue_budget_over_the_instruction_count():
    ops, per_clk, _, _ = bench.ops_per_update(bench.PROFILE_SUMMARY)
    peak, basis = bench.issue_peak(152, 2070.0, bench.PROFILE_SUMMARY)
    assert math.isclose(peak, 152 * per_clk * 2070e6 / ops / 1e9, rel_tol=1e-12)
    assert "152 SMs" in basis


def test_helpers():
    assert bench.tail_kernel(10, None) is None
    assert bench.tail_kernel(10, {"words": 16, "threads": 320, "ctas_per_sm": 2}) == "k_sweep<10,16,320,2>"
    assert bench.reduce_over_ranks(3.5, 1e9) == (3.5, 1e9)
