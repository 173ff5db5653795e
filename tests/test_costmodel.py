"""The algorithmic flop counts behind the bench's roofline figures
(paper_2207_00426_gb300.costmodel): the level shapes follow the library's
plan, the upper levels count the work-efficient number of combines whatever
the bracketing, and the refinement passes count their mean-only kernels at
their own cost exactly where the library takes that form."""
import numpy as np
import pytest

from paper_2207_00426_gb300 import costmodel as CM


def _leaf_chunks(lengths, leaf):
    return sum((n + leaf - 1) // leaf for n in lengths)


def test_levels_of_the_benchmark_sequence():
    """n = 1e5, leaf 3, adaptive radix: 33334 leaf chunks, then 32-item
    chunk levels until one item is left (the shape of the benchmark)."""
    lv = CM._levels([100_000], 3, 0)
    assert [len(l) for l in lv] == [33334, 1042, 33, 2, 1]
    assert sum(lv[0]) == 100_000 and max(lv[0]) == 3
    assert all(max(l) <= 32 for l in lv[1:])


def test_fold_levels_above_the_chunk_scan_limit():
    """A level of more than FOLD_ABOVE_ITEMS items is folded 4 at a time."""
    lv = CM._levels([2 ** 20], 4, 0)
    assert len(lv[1]) == 2 ** 18 // 4 and max(lv[1]) == 4
    assert max(lv[2]) == 32


@pytest.mark.parametrize("lengths", [[100_000], [5, 1, 700, 33, 96], [3000] * 7])
def test_upper_levels_count_one_combine_per_merged_item(lengths):
    """However the tree is bracketed, reducing the leaf aggregates of each
    sequence to one item takes (items - 1) combines per sequence."""
    leaf = CM.default_leaf(sum(lengths))
    f = CM.ipls_kernel_flops(lengths, leaf=leaf)
    merges = _leaf_chunks(lengths, leaf) - len(lengths)
    up = f.get("filter_up", (0.0, 0))
    assert up[0] * up[1] == pytest.approx(merges * CM.filter_combine(5))
    down = f.get("filter_down", (0.0, 0))
    assert down[0] * down[1] == pytest.approx(merges * CM.filter_apply(5))


def test_mean_only_combine_count():
    """filter_combine_means: three products with the lower factor U_i and
    two with Z_j (n(n+1)/2 FMAs each), three full n x n products (A_j(I -
    U_i G^T), G, A_i^T) and five vector sums."""
    for nx in (1, 3, 5):
        tri = nx * (nx + 1)
        assert CM.filter_combine_means(nx) == 5 * tri + 3 * 2 * nx * nx + 5 * nx
    assert CM.filter_combine_means(5) == 325
    assert CM.filter_combine_means(5) < CM.filter_combine(5) / 10


def _total(f, key):
    a, n = f[key]
    return a * n


def test_refinement_counts_the_mean_only_filter_levels():
    """One refinement pass at n = 1e5: the filter scan runs twice; in the
    second pass the levels of at most CS3_MAX_CHUNKS chunks (33 chunks, then
    the top's 33 items: 1009 + 32 combines) take the mean-only cost."""
    n = [100_000]
    f0 = CM.ipls_kernel_flops(n, leaf=3)
    f1 = CM.ipls_kernel_flops(n, leaf=3, refine=1)
    fc, fm = CM.filter_combine(5), CM.filter_combine_means(5)
    small = (1042 - 33) + (33 - 2) + (2 - 1)
    expect = 2 * _total(f0, "filter_up") - small * (fc - fm)
    assert _total(f1, "filter_up") == pytest.approx(expect)
    # the rest of the filter scan runs in full twice
    for k in ("filter_leaf_up", "filter_down", "filter_leaf_down"):
        assert _total(f1, k) == pytest.approx(2 * _total(f0, k))
    # the smoother once in full, once mean-only
    for k in ("smoother_leaf_up", "smoother_up", "smoother_down", "smoother_leaf_down"):
        assert _total(f0, k) < _total(f1, k) < 2 * _total(f0, k)


@pytest.mark.parametrize("case", ["many sequences", "small state"])
def test_refinement_without_mean_only_filter_levels(case):
    """Beyond FMEANS_MAX_SEQS sequences, or below FMEANS_MIN_NX state
    entries, the library runs the refinement's filter scan in full."""
    if case == "many sequences":
        lengths, kw = [3000] * (CM.FMEANS_MAX_SEQS + 1), {}
    else:
        lengths, kw = [3000] * 4, {"nx": 1, "ny": 1}
    f0 = CM.ipls_kernel_flops(lengths, **kw)
    f1 = CM.ipls_kernel_flops(lengths, refine=1, **kw)
    assert _total(f1, "filter_up") == pytest.approx(2 * _total(f0, "filter_up"))


def test_iteration_flops_fall_with_the_mean_only_passes():
    """A refinement pass costs less than a first pass (no Tria in its
    smoother or its filter's small levels) but more than nothing."""
    n = [100_000]
    it0 = CM.ipls_iteration_flops(n, leaf=3)
    it1 = CM.ipls_iteration_flops(n, leaf=3, refine=1)
    slr = _total(CM.ipls_kernel_flops(n, leaf=3), "ct_slr")
    assert it0 < it1 < 2 * it0 - slr
    assert np.isfinite(it1)
