"""Warp orders of the packings (host only, no GPU).

SG_PACK_CLASS keeps the packer's class-grouped order (the identity);
SG_PACK_INTERLEAVE places warp i of a run of n warps of one warp class at the
fractional position (2 i + 1) / (2 n).  The bound checked here follows from
that rule alone: if x is the position of the k-th warp of the merged order,
a run of n_c warps has floor(x n_c + 1/2) warps at or before x, so every run
holds within 1/2 of x n_c of the first k warps, their sum k lies within m/2
of x NW (m runs), and so every run's share of any prefix of k warps is within
1/2 + m/2 of its proportional share k n_c / NW.
"""
import numpy as np
import pytest

from paper_2310_04676_gb300 import sg, workloads as W


@pytest.fixture(scope="module")
def lib():
    return sg.load_library()


def _runs(kinds):
    """Run sizes (warps) of the class-grouped order for the kinds of the
    mixed batch: 7R two-arm envs (lane pairs), 7R, 7P, 4R, each run padded to
    whole warps."""
    n14 = kinds.count("14B")
    sizes = [-(-2 * n14 // 32), -(-kinds.count("7R") // 32), -(-kinds.count("7P") // 32),
             -(-kinds.count("4R") // 32)]
    return [s for s in sizes if s]


@pytest.mark.parametrize("E", [1000, 5000])
def test_interleave_order_is_a_proportional_permutation(lib, E):
    kinds = W.mixed_kinds(E, W.C3_FRACTIONS)
    d = W.make_desc(kinds)
    sizes = _runs(kinds)
    NW = sum(sizes)
    assert sg.plan(d)["num_slots"] == 32 * NW
    ident = sg.plan_packing(d, sg.PACK_CLASS)
    assert np.array_equal(ident, np.arange(NW))
    order = sg.plan_packing(d, sg.PACK_INTERLEAVE)
    assert sorted(order.tolist()) == list(range(NW))
    run_of = np.repeat(np.arange(len(sizes)), sizes)[order]
    m = len(sizes)
    counts = np.zeros(m)
    worst = 0.0
    for k in range(1, NW + 1):
        counts[run_of[k - 1]] += 1
        worst = max(worst, float(np.abs(counts - k * np.array(sizes) / NW).max()))
    assert worst <= 0.5 + m / 2
    # within each run the class-grouped order (caller order) is kept
    for r in range(m):
        pos = order[run_of == r]
        assert np.all(np.diff(pos) > 0)
    # a mixed prefix: the first m warps come from m different runs
    assert len(set(run_of[:m].tolist())) == m


def test_homogeneous_batch_has_one_order(lib):
    d = W.make_desc(["7R"] * 300)
    assert np.array_equal(sg.plan_packing(d, sg.PACK_INTERLEAVE), sg.plan_packing(d, sg.PACK_CLASS))


def test_unknown_packing_is_rejected(lib):
    d = W.make_desc(["7R"] * 64)
    with pytest.raises(sg.SgError) as e:
        sg.plan_packing(d, 7)
    assert e.value.status == sg.SG_ERR_INVALID_ARG
