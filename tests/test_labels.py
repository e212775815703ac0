"""Sub-subdomains given per element (bddc_partition.piece): the library's
host classification against the oracle's (Section 3: objects are connected
sets of interface nodes with equal sets of surrounding sub-subdomains, typed
by the size of that set), on the synthetic channels sub-partition of
Section 5.2 and on box labels, where it must reproduce the box rule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import objects, partition  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    import paper_2001_07289_gb300.bddc as m
    return m


def oracle_counts(nx, ny, nz, sub, piece, sel):
    o = objects.classify(nx, ny, nz, sub, piece)
    keep = objects.select(o, sel)
    k = o.kind[keep]
    return {"n_coarse": len(keep), "n_vertices": int(np.sum(k == 0)), "n_edges": int(np.sum(k == 1)),
            "n_faces": int(np.sum(k == 2))}


@pytest.mark.parametrize("sel", ["vef", "f", "ve", "ef"])
@pytest.mark.parametrize("n,parts,per_axis", [(20, 2, 2), (24, 3, 3), (40, 4, 3)])
def test_channel_objects_match_oracle(gb, n, parts, per_axis, sel):
    p = inputs.channels_problem(n, parts, 4, per_axis=per_axis, selection=sel)
    sub, _ = partition.box_labels(n, n, n, p.cuts, n)
    a = gb.analyze(n, n, n, p.cuts, p.L, selection=sel, piece=p.piece)
    want = oracle_counts(n, n, n, sub, p.piece, sel)
    for k, v in want.items():
        assert a[k] == v, (k, a[k], v)


@pytest.mark.parametrize("case", [(14, 11, 9, [[5, 9], [4], [3, 6]], 3), (12, 12, 12, [[4, 8]] * 3, 2),
                                  (16, 16, 16, [[8]] * 3, 4)])
@pytest.mark.parametrize("sel", ["vef", "vf", "f"])
def test_box_labels_reproduce_box_rule(gb, case, sel):
    nx, ny, nz, cuts, L = case
    _, piece = partition.box_labels(nx, ny, nz, cuts, L)
    a = gb.analyze(nx, ny, nz, cuts, L, selection=sel, piece=piece)
    b = gb.analyze(nx, ny, nz, cuts, L, selection=sel)
    for k in ("n_coarse", "n_vertices", "n_edges", "n_faces", "max_local_coarse"):
        assert a[k] == b[k], k


def test_label_errors(gb):
    n = 8
    cuts = [[4]] * 3
    lab = np.zeros(n ** 3, dtype=np.int64)     # one label across all subdomains
    with pytest.raises(gb.BddcError) as e:
        gb.analyze(n, n, n, cuts, 4, piece=lab)
    assert e.value.code == gb.BDDC_ERR_ARG and "spans two subdomains" in str(e.value)
    _, piece = partition.box_labels(n, n, n, cuts, 4)
    piece = piece.copy()
    piece[0] = -1
    with pytest.raises(gb.BddcError):
        gb.analyze(n, n, n, cuts, 4, piece=piece)
    with pytest.raises(ValueError):
        gb.analyze(n, n, n, cuts, 4, piece=piece[:-1])


@pytest.mark.parametrize("n,parts,ell,straddle", [(20, 2, 6, True), (20, 2, 6, False), (24, 3, 4, False)])
@pytest.mark.parametrize("sel", ["f", "vef", "v"])
def test_paths_with_labels_match_oracle(gb, n, parts, ell, straddle, sel):
    """The acceptable-path check on label-given sub-subdomains (channels),
    library against oracle: counts exactly, smallest quality to rounding."""
    from oracle import paths
    cuts = [inputs.uniform_cuts(n, parts)] * 3
    if straddle:   # one bar along x across the cut plane y = n/2 (quality 10^-ell under faces only)
        m = np.zeros((n, n, n), dtype=bool)
        m[4:6, n // 2 - 1:n // 2 + 1, :] = True
        mask = m.reshape(-1)
    else:
        mask = inputs.channel_mask(n, n, n, 3, 2, 11, cuts)
    piece = inputs.material_pieces(n, n, n, cuts, mask)
    alpha = np.where(mask, 10.0 ** ell, 1.0)
    got = gb.acceptable_paths(n, n, n, cuts, n, alpha=alpha, selection=sel, piece=piece)
    sub, _ = partition.box_labels(n, n, n, cuts, n)
    ref = paths.acceptable_paths(n, n, n, sub, piece, alpha, sel)
    for k in ("n_pieces", "n_pairs", "n_direct", "n_without_path"):
        assert got[k] == ref[k], (k, got[k], ref[k])
    assert got["min_ratio"] == pytest.approx(ref["min_ratio"], rel=1e-12)
