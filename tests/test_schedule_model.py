"""The schedule model of Sec. 3.2 in the library's host code, pinned to the
values the paper prints (tests/golden/paper_schedule_tables.json).  CPU only:
these entry points touch no GPU."""
import json
import os

import pytest

from paper_1505_08067_gb300 import gbfft as g

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_schedule_tables.json")))


def _cost(table):
    return [table["2"], table["4"], table["8"]]


@pytest.mark.parametrize("n", sorted(GOLD["mixed_radix_counts"]["printed"], key=int))
def test_schedule_counts_match_paper_table(n):
    printed, runs = GOLD["mixed_radix_counts"]["printed"][n]
    expect = GOLD["mixed_radix_counts"]["corrected"].get(n, printed)
    log2n = int(n).bit_length() - 1
    assert g.fft_schedule_count(log2n, [1, 2, 3]) == expect
    assert runs == 3 * (log2n - 1)          # stage benchmark runs, as the text states


def test_count_brute_force_small():
    """Compositions of log2 N into parts {1,2,3} enumerated directly."""
    def comps(m):
        if m == 0:
            return 1
        return sum(comps(m - p) for p in (1, 2, 3) if p <= m)
    for m in range(0, 13):
        assert g.fft_schedule_count(m, [1, 2, 3]) == comps(m)
    assert g.fft_schedule_count(5, [1, 2, 3]) == 13        # the 2^5 digraph of Sec. 3.2
    assert g.fft_schedule_count(10, [1, 2, 3, 4]) > g.fft_schedule_count(10, [1, 2, 3])


@pytest.mark.parametrize("gpu", ["ivb", "hsw"])
def test_path_costs_reproduce_printed_ratios(gpu):
    cost = _cost(GOLD["stage_costs"][gpu])
    c8882 = g.fft_schedule_path_cost(10, [1, 2, 3], cost, [8, 8, 8, 2])
    c4884 = g.fft_schedule_path_cost(10, [1, 2, 3], cost, [4, 8, 8, 4])
    naive = g.fft_schedule_path_cost(10, [1, 2, 3], cost, [2] * 10)
    r = GOLD["ratios"][gpu]
    assert round(c8882 / c4884, 2) == r["8882_over_4884"]
    assert round(naive / c4884, 2) == r["naive_over_4884"]
    if "naive_over_8882" in r:
        assert round(naive / c8882, 2) == r["naive_over_8882"]
    expect = {"ivb": (21932, 20970, 27552), "hsw": (20770, 19206, 26072)}[gpu]
    assert (c8882, c4884, naive) == expect


@pytest.mark.parametrize("gpu,best", [("ivb", 19785), ("hsw", 18218)])
def test_shortest_path_on_paper_tables(gpu, best):
    cost = _cost(GOLD["stage_costs"][gpu])
    path, total = g.fft_schedule_shortest_path(10, [1, 2, 3], cost)
    assert path == [8, 8, 4, 4] and total == best
    # brute force over all 274 schedules confirms it is the minimum
    def all_paths(s):
        if s == 10:
            yield []
            return
        for lg in (1, 2, 3):
            if s + lg <= 10 and cost[lg - 1][s] is not None:
                for rest in all_paths(s + lg):
                    yield [1 << lg] + rest
    costs = [g.fft_schedule_path_cost(10, [1, 2, 3], cost, p) for p in all_paths(0)]
    assert len(costs) == 274 and min(costs) == best


def test_shortest_path_rejects_bad_input():
    with pytest.raises(g.GbfftError):
        g.fft_schedule_shortest_path(4, [3], [[1, 1, 1, 1]])          # 8 never reaches 16
    with pytest.raises(g.GbfftError):
        g.fft_schedule_path_cost(4, [1, 2], [[1] * 4, [1] * 4], [4, 2])  # sums to 2^3


@pytest.mark.parametrize("gpu", ["ivb", "hsw"])
def test_eq1_bandwidth_bound(gpu):
    e = GOLD["eq1"][gpu]
    v = g.fft_bandwidth_bound_gflops(GOLD["eq1"]["n"], e["bandwidth_gbs"])
    assert v == e["formula_gflops"]
    assert round(v) in (e["printed_gflops"], e["printed_gflops"] - 1)
    # the GB300 minimum-traffic form: one read and one write per pass
    assert g.fft_bandwidth_bound_gflops(1024, 6792.1, 16, 1) == pytest.approx(5 * 10 * 6792.1 / 16)
