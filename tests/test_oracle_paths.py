"""Pins of the oracle's acceptable-path check (remark after Theorem 1).

- A hand-worked case: four subdomains around one vertical edge of a 4x4x2
  mesh, one sub-subdomain each, rho = 1, 0.01, 0.1, 1.  The four face pairs
  share a face object; the two diagonal pairs share only the edge.  With faces
  only, the diagonal pair (0, 3) goes through piece 1 (rho 0.01) or piece 2
  (rho 0.1): quality 0.1; the pair (1, 2) has min(rho) = 0.01 at its ends and
  quality 1.
- The remark's claim: all-edge or all-face selections leave no pair without
  an acceptable path (constant coefficient: every quality 1).
- Vertices only: across Gamma no link exists unless a contact is all primal,
  so at L = 2 only the pairs touching at one vertex are direct and every
  other pair lacks a path; at L = 1 every interface node is a vertex, every
  contact is primal and every pair is direct.
"""
import numpy as np
import pytest

from oracle import partition, paths


def hand_case(selection):
    nx, ny, nz = 4, 4, 2
    sub, piece = partition.box_labels(nx, ny, nz, [[2], [2], []], 4)
    rho = np.array([1.0, 0.01, 0.1, 1.0])
    return paths.acceptable_paths(nx, ny, nz, sub, piece, rho[piece], selection)


def test_hand_case_faces_only():
    r = hand_case("f")
    assert (r["n_pieces"], r["n_pairs"], r["n_direct"], r["n_without_path"]) == (4, 6, 4, 0)
    assert r["quality"] == {(0, 3): pytest.approx(0.1), (1, 2): 1.0}
    assert r["min_ratio"] == pytest.approx(0.1)


@pytest.mark.parametrize("sel", ["vef", "ve", "ef"])
def test_hand_case_edges_direct(sel):
    r = hand_case(sel)
    assert (r["n_pairs"], r["n_direct"], r["n_without_path"], r["min_ratio"]) == (6, 6, 0, 1.0)


def test_hand_case_vertices_only():
    # both ends of the shared edge lie on the Dirichlet boundary: no vertex object
    r = hand_case("v")
    assert (r["n_pairs"], r["n_direct"], r["n_without_path"]) == (6, 0, 6)


CASES = [
    (12, 12, 12, [[4, 8]] * 3, 2),
    (12, 12, 12, [[4, 8]] * 3, 3),
    (14, 11, 9, [[5, 9], [4], [3, 6]], 3),
    (14, 11, 9, [[5, 9], [4], [3, 6]], 2),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("sel", ["vef", "ve", "ef", "f"])
def test_all_edges_or_all_faces_give_paths(case, sel):
    nx, ny, nz, cuts, L = case
    sub, piece = partition.box_labels(nx, ny, nz, cuts, L)
    r = paths.acceptable_paths(nx, ny, nz, sub, piece, None, sel)
    assert r["n_pairs"] > 0 and r["n_without_path"] == 0 and r["min_ratio"] == 1.0


def test_vertices_only():
    """L = 2 on 12^3 with 3^3 subdomains: 6 pieces per axis, 5^3 interior
    piece corners, each with 4 body-diagonal pairs touching only there; the
    pair crosses a cut when one of the corner's indices is a cut (1 or 3 of
    0..4): 4 (125 - 27) = 392 pairs whose whole contact is one primal vertex.
    Every other pair lacks a path."""
    sub, piece = partition.box_labels(12, 12, 12, [[4, 8]] * 3, 2)
    r = paths.acceptable_paths(12, 12, 12, sub, piece, None, "v")
    assert r["n_direct"] == 392 and r["n_without_path"] == r["n_pairs"] - 392 > 0
    sub, piece = partition.box_labels(12, 12, 12, [[4, 8]] * 3, 1)
    r = paths.acceptable_paths(12, 12, 12, sub, piece, None, "v")
    assert r["n_direct"] == r["n_pairs"] > 0 and r["n_without_path"] == 0


def test_quality_is_the_best_path_bottleneck_brute_force():
    """Every simple path enumerated on a 3x3x1 arrangement of one-piece
    subdomains with random rho, faces only: each pair's quality is the best
    bottleneck over its paths."""
    import itertools
    nx, ny, nz = 6, 6, 2
    sub, piece = partition.box_labels(nx, ny, nz, [[2, 4], [2, 4], []], 2)
    rng = np.random.default_rng(5)
    rho = 10.0 ** rng.uniform(-3, 0, piece.max() + 1)
    r = paths.acceptable_paths(nx, ny, nz, sub, piece, rho[piece], "f")
    # links: subdomains sharing a face (grid neighbours on the 3 x 3 layout)
    pos = {k: (k % 3, k // 3) for k in range(9)}
    nb = {k: [j for j in range(9) if abs(pos[k][0] - pos[j][0]) + abs(pos[k][1] - pos[j][1]) == 1] for k in range(9)}

    def best(i, j):
        out, stack = 0.0, [(i, (i,))]
        while stack:
            u, path = stack.pop()
            if u == j:
                out = max(out, min(rho[list(path)]))
                continue
            for w in nb[u]:
                if w not in path:
                    stack.append((w, path + (w,)))
        return min(1.0, out / min(rho[i], rho[j]))

    diag = [(i, j) for i, j in itertools.combinations(range(9), 2)
            if abs(pos[i][0] - pos[j][0]) == 1 and abs(pos[i][1] - pos[j][1]) == 1]
    assert sorted(r["quality"]) == sorted(diag)
    for (i, j), q in r["quality"].items():
        assert q == pytest.approx(best(i, j), rel=1e-12)


def test_channels_need_paths_through_the_channels():
    """Channels of contrast 10^6 on 20^3 with 2^3 subdomains, one channel
    piece per subdomain (Section 5.2).  A bar straddling the cut plane
    parallel to it meets its continuation in the diagonal subdomain only along
    an edge: with faces only, that channel pair's best path crosses the
    background, quality 1e-6.  The same bar inside a slab leaves every pair a
    path through the channel (quality 1)."""
    from paper_2001_07289_gb300 import inputs
    n, cuts = 20, [[10]] * 3
    sub, _ = partition.box_labels(n, n, n, cuts, n)
    for y0, want in ((9, 1e-6), (4, 1.0)):   # bar along x at y in [y0, y0+2), z in [4, 6)
        mask = np.zeros((n, n, n), dtype=bool)
        mask[4:6, y0:y0 + 2, :] = True
        mask = mask.reshape(-1)
        piece = inputs.material_pieces(n, n, n, cuts, mask)
        alpha = np.where(mask, 1e6, 1.0)
        r = paths.acceptable_paths(n, n, n, sub, piece, alpha, "f")
        assert r["n_without_path"] == 0
        assert r["min_ratio"] == pytest.approx(want, rel=1e-12)
