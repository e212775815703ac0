"""The library's acceptable-path check (bddc_acceptable_paths, host code)
against the oracle's on tensor sub-partitions, selections and log-uniform
coefficients: counts exactly, the smallest quality to rounding, and the
reported worst pair has that quality (or no path) in the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import partition, paths  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    import paper_2001_07289_gb300.bddc as m
    return m


CASES = [
    (4, 4, 2, [[2], [2], []], 4),
    (12, 12, 12, [[4, 8]] * 3, 2),
    (12, 12, 12, [[4, 8]] * 3, 1),
    (14, 11, 9, [[5, 9], [4], [3, 6]], 3),
    (16, 12, 10, [[5, 11], [6], [4]], 2),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("sel", ["vef", "ve", "vf", "v", "f", "ef"])
@pytest.mark.parametrize("coef", ["one", "loguniform"])
def test_paths_match_oracle(gb, case, sel, coef):
    nx, ny, nz, cuts, L = case
    alpha = None if coef == "one" else inputs.alpha_loguniform(nx, ny, nz, -3, 3, 7)
    got = gb.acceptable_paths(nx, ny, nz, cuts, L, alpha=alpha, selection=sel)
    sub, piece = partition.box_labels(nx, ny, nz, cuts, L)
    ref = paths.acceptable_paths(nx, ny, nz, sub, piece, alpha, sel)
    for k in ("n_pieces", "n_pairs", "n_direct", "n_without_path"):
        assert got[k] == ref[k], (k, got[k], ref[k])
    assert got["min_ratio"] == pytest.approx(ref["min_ratio"], rel=1e-12)
    if ref["n_pairs"] > ref["n_direct"]:
        q = ref["quality"][tuple(sorted(got["worst_pair"]))]
        if ref["n_without_path"]:
            assert q is None
        else:
            assert q == pytest.approx(ref["min_ratio"], rel=1e-12)
    else:
        assert got["worst_pair"] == [-1, -1]


def test_paths_argument_errors(gb):
    with pytest.raises(ValueError):
        gb.acceptable_paths(8, 8, 8, [[4]] * 3, 2, alpha=np.ones(10))
    with pytest.raises(gb.BddcError) as e:
        gb.acceptable_paths(8, 8, 8, [[4]] * 3, 0)
    assert e.value.code == gb.BDDC_ERR_ARG
