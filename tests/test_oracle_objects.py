"""Pins of the oracle's partition, sub-partition and (sub)object classification
(Section 3; Table 1 coarse sizes)."""
import numpy as np
import pytest

from oracle import objects, partition
from paper_2001_07289_gb300 import inputs
from tests.golden import read as golden

T1 = golden.table1_coarse_sizes()


def count_objects(n, parts, L):
    cuts = [inputs.uniform_cuts(n, parts)] * 3
    sub, piece = partition.box_labels(n, n, n, cuts, L)
    return objects.classify(n, n, n, sub, piece)


def tensor_counts(m, s):
    """Closed form for m^3 box subdomains each cut into s^3 pieces, n = m s
    pieces per axis: faces 3(m-1)n^2, edges 3n((n-1)^2-(n-m)^2), vertices
    (n-1)^3-(n-m)^3 (a face sits on one Theta plane and two piece intervals; an
    edge on two piece cut planes of which at least one is a Theta plane; a
    vertex on three)."""
    n = m * s
    return dict(faces=3 * (m - 1) * n * n,
                edges=3 * n * ((n - 1) ** 2 - (n - m) ** 2),
                vertices=(n - 1) ** 3 - (n - m) ** 3)


def test_subdivision_rule():
    assert partition.subdivide(0, 12, 4) == [4, 8]
    assert partition.subdivide(0, 12, 5) == [4, 8]
    assert partition.subdivide(3, 10, 4) == [6]
    assert partition.subdivide(0, 7, 2) == [1, 3, 5]
    assert partition.subdivide(0, 5, 9) == []


@pytest.mark.parametrize("m,s,L", [(2, 2, 3), (3, 2, 3), (3, 3, 3), (4, 1, 4), (2, 4, 3)])
def test_counts_match_closed_form(m, s, L):
    n_el = m * s * L
    o = count_objects(n_el, m, L)
    assert o.counts() == tensor_counts(m, s)


@pytest.mark.parametrize("m,s", [(2, 2), (3, 3), (2, 5)])
def test_total_count_one_node_intervals(m, s):
    """With L = 2 every interval holds one node; the object count is unchanged,
    and so are the type counts: a face shared by two sub-subdomains stays a
    face when it is a single node (types come from the sub-subdomain lists,
    not from the object's extent)."""
    o = count_objects(m * s * 2, m, 2)
    assert len(o) == sum(tensor_counts(m, s).values())
    assert o.counts() == tensor_counts(m, s)


def test_workload_poisson16_counts():
    """16^3, 2^3 subdomains, L=4: 127 coarse DOFs (48 faces, 60 edges, 19
    vertices) and 37 on every subdomain."""
    p = inputs.workload(0)
    sub, piece = partition.box_labels(16, 16, 16, p.cuts, p.L)
    o = objects.classify(16, 16, 16, sub, piece)
    assert len(o) == 127
    assert o.counts() == dict(vertices=19, edges=60, faces=48)
    per_sub = np.bincount(np.concatenate(o.subdomains))
    assert (per_sub == 37).all()


def test_table1_k4_true_size():
    """Table 1, k=4 (40^3 hexahedra, 10^3 subdomains, L/h=4): 5,859 for both
    BDDC(vef) and BDDC-SO(vef)."""
    assert len(count_objects(40, 10, 4)) == T1[("BDDC-SO(vef)", 4)] == T1[("BDDC(vef)", 4)]


def test_table1_k8_true_size():
    """Table 1, k=8 (80^3, L/h=4): BDDC-SO(vef) has 32,319 coarse DOFs and
    BDDC(vef) (no sub-partition, L = k) 5,859."""
    assert len(count_objects(80, 10, 4)) == T1[("BDDC-SO(vef)", 8)]
    assert len(count_objects(80, 10, 8)) == T1[("BDDC(vef)", 8)]


@pytest.mark.parametrize("k", [16, 24])
def test_table1_large_k_reduced_mesh(k):
    """Table 1, k=16 and k=24 at L/h=4: k/4 pieces per subdomain side.  The
    objects depend only on the arrangement of pieces, so the count is taken on
    the mesh with the same pieces two elements wide (one node per interval)."""
    s = k // 4
    assert len(count_objects(10 * s * 2, 10, 2)) == T1[("BDDC-SO(vef)", k)]


def test_object_keys_and_subdomains():
    o = count_objects(12, 2, 3)
    for nodes, kind, subs, key in zip(o.nodes, o.kind, o.subdomains, o.key):
        assert len(subs) in (2, 4, 8)
        # every node of an object has the same pieces
        for v in nodes:
            pcs = o.node_pieces[v][o.node_pieces[v] >= 0]
            assert np.array_equal(pcs, key)
        assert len(key) == 2 ** (3 - kind)
