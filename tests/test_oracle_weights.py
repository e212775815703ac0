"""Pins of the weighting E (eq. W and Remark 1)."""
import numpy as np

from oracle import bddc, objects, partition, weights
from paper_2001_07289_gb300 import inputs
from tests.golden import read as golden


def _fig1_labels(nz=2):
    """Figure 1 extruded in z: 20x20 cells, Theta = 2x2 (cut at 10), Omega_1 =
    [0,10]^2 split into the square Omega-hat_2 = [5,10]^2 and the L-shaped rest
    Omega-hat_1; Omega_2 = [0,10]x[10,20] split into [5,10]x[10,16] (hat 4) and
    the rest (hat 3); Omega_3, Omega_4 split by x = 15 (hats 5, 6 and 7, 8).
    Labels are 0-based (hat j -> j-1, Omega_i -> i-1)."""
    n = 20
    sub = np.zeros((nz, n, n), dtype=np.int64)
    piece = np.zeros((nz, n, n), dtype=np.int64)
    for j in range(n):
        for i in range(n):
            right, top = i >= 10, j >= 10
            sub[:, j, i] = {(0, 0): 0, (0, 1): 1, (1, 0): 2, (1, 1): 3}[(right, top)]
            if not right and not top:
                piece[:, j, i] = 1 if (i >= 5 and j >= 5) else 0
            elif not right and top:
                piece[:, j, i] = 3 if (i >= 5 and j < 16) else 2
            elif right and not top:
                piece[:, j, i] = 4 if i < 15 else 5
            else:
                piece[:, j, i] = 6 if i < 15 else 7
    return sub.ravel(), piece.ravel()


def test_figure1_weight_two_thirds():
    """delta_1(xi) = card{1,2}/card{1,2,5} = 2/3 at xi = (10, 5), where the
    multiplicity weight is 1/2."""
    nz = 2
    sub, piece = _fig1_labels(nz)
    o = objects.classify(20, 20, nz, sub, piece)
    parent = weights.piece_parent(sub, piece)
    xi = 10 + 21 * (5 + 21 * 1)
    g = golden.fig1()
    assert weights.delta(xi, 0, o.node_pieces, parent) == g["delta_1"]
    assert abs(weights.delta(xi, 2, o.node_pieces, parent) - (1 - g["delta_1"])) < 1e-15
    assert 1 / np.sum(o.node_subs[xi] >= 0) == g["multiplicity_weight"]
    # the point is a one-node object with key {hat1, hat2, hat5}
    k = [i for i, nodes in enumerate(o.nodes) if xi in nodes]
    assert len(k) == 1 and list(o.key[k[0]]) == [0, 1, 4] and len(o.nodes[k[0]]) == 1


def _check_unity(B):
    tot = np.zeros(B.nn)
    for s in B.subs:
        np.add.at(tot, s.nodes[s.gamma_loc], s.delta)
    assert np.abs(tot[B.gamma] - 1.0).max() < 1e-14


def test_partition_of_unity_card_and_rho():
    p = inputs.box_problem(12, 12, 12, [[4, 8], [6], [3, 9]], 2,
                           alpha=inputs.alpha_blocks(12, 12, 12, 2, 1e4, 0.4, 3))
    for w in ("card", "rho"):
        p.weights = w
        _check_unity(bddc.build(p))


def test_tensor_card_weights_are_inverse_multiplicity():
    p = inputs.box_problem(12, 12, 12, [[4, 8]] * 3, 2)
    B = bddc.build(p)
    for s in B.subs:
        mult = np.sum(B.objs.node_subs[s.nodes[s.gamma_loc]] >= 0, axis=1)
        assert np.abs(s.delta - 1.0 / mult).max() < 1e-15


def test_rho_weights_follow_remark1():
    """On a face between a piece of alpha=1e4 and one of alpha=1 the high
    side gets 1e4/(1e4+1)."""
    n = 8
    a = np.ones(n ** 3).reshape(n, n, n)
    a[:, :, :4] = 1e4                      # x < 4 high
    p = inputs.box_problem(n, n, n, [[4], [], []], 4, alpha=a.ravel(), weights="rho")
    B = bddc.build(p)
    node = 4 + 9 * (3 + 9 * 3)            # on the x=4 face, inside the face
    for i, s in enumerate(B.subs):
        loc = np.flatnonzero(s.nodes[s.gamma_loc] == node)
        want = 1e4 / (1e4 + 1) if i == 0 else 1 / (1e4 + 1)
        assert abs(s.delta[loc[0]] - want) < 1e-15
