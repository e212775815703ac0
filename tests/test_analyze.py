"""The library's own host-side classification and coarse elimination plan
(bddc_analyze, no GPU) against the paper's Table 1 and the oracle."""
import pytest

pytest.importorskip("torch")

from oracle import objects, partition  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402
from tests.golden import read as golden  # noqa: E402


@pytest.fixture(scope="module")
def gb():
    import os
    from paper_2001_07289_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    import paper_2001_07289_gb300.bddc as gb
    return gb


@pytest.mark.parametrize("k", [4, 8, 16, 24])
def test_table1_coarse_sizes_full_size(gb, k):
    """Table 1: (10k)^3 hexahedra, 10^3 subdomains, L/h = 4 (BDDC-SO(vef)) and
    L = k (BDDC(vef)), counted on the true meshes."""
    t1 = golden.table1_coarse_sizes()
    n = 10 * k
    cuts = [inputs.uniform_cuts(n, 10)] * 3
    assert gb.analyze(n, n, n, cuts, 4)["n_coarse"] == t1[("BDDC-SO(vef)", k)]
    if ("BDDC(vef)", k) in t1:
        assert gb.analyze(n, n, n, cuts, k)["n_coarse"] == t1[("BDDC(vef)", k)]


def test_type_counts_closed_form(gb):
    # m = 3 subdomains per axis, s = 3 pieces each (L = 4, w = 12): n = 9
    a = gb.analyze(36, 36, 36, [[12, 24]] * 3, 4)
    m, n = 3, 9
    assert a["n_faces"] == 3 * (m - 1) * n * n
    assert a["n_edges"] == 3 * n * ((n - 1) ** 2 - (n - m) ** 2)
    assert a["n_vertices"] == (n - 1) ** 3 - (n - m) ** 3


@pytest.mark.parametrize("case", [
    (16, 16, 16, [[8], [8], [8]], 4),
    (14, 11, 9, [[5, 9], [4], [3, 6]], 3),
    (10, 9, 8, [[3, 7], [2, 5], [4]], 1),
    (8, 8, 8, [[1, 2, 6], [4], [7]], 2),
    (12, 6, 6, [[4, 8], [], []], 4),
    (8, 8, 8, [[], [], []], 4),
    (20, 20, 20, [[3, 8, 12, 17], [5, 10, 15], [7]], 2),
])
def test_counts_match_oracle(gb, case):
    nx, ny, nz, cuts, L = case
    sub, piece = partition.box_labels(nx, ny, nz, cuts, L)
    o = objects.classify(nx, ny, nz, sub, piece)
    a = gb.analyze(nx, ny, nz, cuts, L)
    assert a["n_coarse"] == len(o)
    assert a["n_sub"] == sub.max() + 1


@pytest.mark.parametrize("m,L", [(2, 4), (4, 4), (4, 2), (8, 4), (3, 3), (16, 2)])
def test_nested_dissection_plan(gb, m, L):
    """Every coarse DOF is a pivot of exactly one front and every child update
    set nests in its parent front (bddc_analyze fails otherwise); the plan does
    far less work than a dense factorisation."""
    n = 12 * m if m <= 8 else 8 * m
    cuts = [inputs.uniform_cuts(n, m)] * 3
    a = gb.analyze(n, n, n, cuts, L)
    nc = a["n_coarse"]
    assert a["n_fronts"] >= 1
    if nc > 2000:
        assert a["coarse_fma"] < (nc ** 3 / 6) / 4


def test_jittered_workload_plan(gb):
    p = inputs.workload(3, L=4)
    a = gb.analyze(p.nx, p.ny, p.nz, p.cuts, 4)
    assert a["n_sub"] == 4096
    assert 150000 < a["n_coarse"] < 260000
    assert a["n_fronts"] > 0


@pytest.mark.parametrize("case", [
    (14, 11, 9, [[5, 9], [4], [3, 6]], 3),
    (20, 20, 20, [[3, 8, 12, 17], [5, 10, 15], [7]], 2),
    (36, 36, 36, [[12, 24]] * 3, 4),
])
@pytest.mark.parametrize("sel", ["ve", "vf", "v", "f", "ef"])
def test_selection_variants_match_oracle(gb, case, sel):
    """Section 5's selection variants: the library's coarse objects are
    exactly the oracle's selected objects, and the type counts are the vef
    counts with the dropped types removed."""
    nx, ny, nz, cuts, L = case
    sub, piece = partition.box_labels(nx, ny, nz, cuts, L)
    o = objects.classify(nx, ny, nz, sub, piece)
    a = gb.analyze(nx, ny, nz, cuts, L, selection=sel)
    full = gb.analyze(nx, ny, nz, cuts, L)
    assert a["n_coarse"] == len(objects.select(o, sel))
    keep = {"ve": ("n_vertices", "n_edges"), "vf": ("n_vertices", "n_faces"), "v": ("n_vertices",),
            "f": ("n_faces",), "ef": ("n_edges", "n_faces")}[sel]
    for key in ("n_vertices", "n_edges", "n_faces"):
        assert a[key] == (full[key] if key in keep else 0)
    assert a["n_coarse"] == sum(full[k] for k in keep)


def test_unknown_selection_rejected(gb):
    with pytest.raises(gb.BddcError) as e:
        gb.analyze(16, 16, 16, [[8]] * 3, 4, selection=6)
    assert e.value.code == gb.BDDC_ERR_ARG