"""bench.py's roofline numerator is the algorithmic FLOP count of the chain
code as it stands: the constants it uses must equal what the counting
scalar measures on the current sources (no GPU)."""
import shutil
import sys

import pytest

from paper_2310_04676_gb300.flops import count as C


def test_bench_constants_match_the_counted_chain_code():
    if not (shutil.which("g++") or shutil.which("c++")):
        pytest.skip("needs a host C++ compiler")
    sys.argv = ["bench"]
    import bench
    got = C.count()
    for pat in ("7R", "7P", "4R"):
        assert got[pat]["substep"] == bench.FLOP_SUBSTEP[pat], pat
        assert got[pat]["tip"] == bench.FLOP_TIP[pat], pat
        assert got[pat]["substep_adjoint"] == bench.FLOP_SUBSTEP_ADJ[pat], pat
        assert got[pat]["tip_vjp"] == bench.FLOP_TIP_VJP[pat], pat
        assert got[pat]["substep_replay"] == bench.FLOP_SUBSTEP_REPLAY[pat], pat


def test_counts_scale_with_the_chain():
    """A 7-joint chain costs more than a 4-joint one, and the adjoint of a
    substep more than the substep it differentiates."""
    if not (shutil.which("g++") or shutil.which("c++")):
        pytest.skip("needs a host C++ compiler")
    got = C.count()
    assert got["4R"]["substep"] < got["7P"]["substep"] < got["7R"]["substep"]
    for pat in got:
        assert got[pat]["substep_adjoint"] > got[pat]["substep_replay"] > got[pat]["substep"]
