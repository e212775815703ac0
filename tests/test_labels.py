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


def test_paths_refuse_labels(gb):
    """The acceptable-path check is written for box sub-subdomains."""
    p = inputs.channels_problem(20, 2, 2, per_axis=2)
    import ctypes as C
    mesh, part, opt, keep = gb._structs(20, 20, 20, 1.0 / 20, p.cuts, p.L, "fp64", "card", 100, False, "f",
                                        piece=p.piece)
    out = gb.Paths()
    code = gb.lib.bddc_acceptable_paths(C.byref(mesh), C.byref(part), C.byref(opt), None, C.byref(out))
    assert code == gb.BDDC_ERR_UNSUPPORTED
