"""Host analysis of the multilevel coarse level (bddc_analyze with
options.ml_block / ml_sub, no GPU): the number of blocks and of level-2
coarse DOFs, with and without level-2 subobjects (Section 6: subobjects at
the coarser levels), against the oracle's three-level preconditioner
(oracle/multilevel.py), which groups the interface coarse DOFs of the coarse
level by the sets of blocks (or sub-blocks) sharing them."""
import pytest

from oracle import bddc as orc, multilevel as ml
from paper_2001_07289_gb300 import inputs
from paper_2001_07289_gb300 import bddc as lib

CASES = [
    # dims, cuts, L, subdomains per axis, g, sub
    ((12, 12, 12), [[3, 6, 9]] * 3, 3, (4, 4, 4), 2, 0),
    ((12, 12, 12), [[3, 6, 9]] * 3, 3, (4, 4, 4), 2, 1),
    ((14, 12, 10), [[3, 7, 10], [4, 8], [5]], 2, (4, 3, 2), 2, 0),
    ((14, 12, 10), [[3, 7, 10], [4, 8], [5]], 2, (4, 3, 2), 2, 1),
    ((15, 15, 15), [[3, 6, 9, 12]] * 3, 3, (5, 5, 5), 3, 2),
    ((15, 15, 15), [[3, 6, 9, 12]] * 3, 3, (5, 5, 5), 4, 3),
]


@pytest.mark.parametrize("dims,cuts,L,nsub,g,sub", CASES)
def test_level2_sizes_match_oracle(dims, cuts, L, nsub, g, sub):
    nx, ny, nz = dims
    p = inputs.box_problem(nx, ny, nz, cuts, L)
    m2 = ml.CoarseBDDC(orc.build(p), nsub, g, "card", sub=sub)
    a = lib.analyze(nx, ny, nz, cuts, L, ml_block=g, ml_sub=sub)
    assert (a["ml_blocks"], a["ml_coarse2"]) == (m2.nblock, m2.ncc)
    assert a["ml_fronts2"] >= (1 if m2.ncc else 0)


def test_level2_subobjects_refine_the_objects():
    """Sub-blocks split the level-2 objects: more level-2 DOFs for smaller
    sub-blocks, the block objects again when the sub-block is the block."""
    args = (15, 15, 15, [[3, 6, 9, 12]] * 3, 3)
    n = [lib.analyze(*args, ml_block=4, ml_sub=s)["ml_coarse2"] for s in (0, 4, 2, 1)]
    assert n[0] == n[1] < n[2] < n[3]


def test_ml_sub_needs_ml_block_host():
    with pytest.raises(RuntimeError, match="ml_sub"):
        lib.analyze(8, 8, 8, [[4]] * 3, 2, ml_sub=1)
