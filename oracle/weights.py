"""The weighting operator E (oracle).

Eq. (W), Section 3: E u(xi) = sum over subdomains Omega_i containing xi of
delta_i(xi) u_i(xi) with

    delta_i(xi) = card{j : Omega-hat_j contains xi, Omega-hat_j inside Omega_i}
                  / card{j : Omega-hat_j contains xi}.

Remark 1 replaces the counts by sums of the (piecewise constant) coefficient
alpha_j of the sub-subdomains:

    delta_i(xi) = sum_{j ∋ xi, j ⊂ Omega_i} alpha_j / sum_{j ∋ xi} alpha_j.

Off the interface delta_i = 1 for the single subdomain holding the node.
"""
from __future__ import annotations

import numpy as np


def piece_alpha(alpha: np.ndarray, piece: np.ndarray) -> np.ndarray:
    """alpha_j of each sub-subdomain: the mean of its element coefficients
    (Remark 1 assumes alpha constant on each piece; then this is that value)."""
    npieces = piece.max() + 1
    s = np.bincount(piece, weights=alpha, minlength=npieces)
    c = np.bincount(piece, minlength=npieces)
    return s / c


def piece_parent(sub: np.ndarray, piece: np.ndarray) -> np.ndarray:
    """Subdomain containing each piece (pieces are unions of elements of one subdomain)."""
    parent = np.full(piece.max() + 1, -1, dtype=np.int64)
    parent[piece] = sub
    return parent


def delta(node: int, i: int, node_pieces: np.ndarray, parent: np.ndarray,
          piece_weight: np.ndarray | None = None) -> float:
    """delta_i(node) of eq. (W) (piece_weight None) or of Remark 1."""
    pcs = node_pieces[node]
    pcs = pcs[pcs >= 0]
    w = np.ones(len(pcs)) if piece_weight is None else piece_weight[pcs]
    inside = parent[pcs] == i
    return float(np.sum(w[inside]) / np.sum(w))


def delta_all(nodes: np.ndarray, i: int, node_pieces: np.ndarray, parent: np.ndarray,
              piece_weight: np.ndarray | None = None) -> np.ndarray:
    """Vectorised delta_i over an array of nodes of subdomain i."""
    pcs = node_pieces[nodes]                       # (m, 8), -1 padded
    valid = pcs >= 0
    safe = np.where(valid, pcs, 0)
    w = np.where(valid, 1.0 if piece_weight is None else piece_weight[safe], 0.0)
    inside = valid & (parent[safe] == i)
    return np.sum(np.where(inside, w, 0.0), axis=1) / np.sum(w, axis=1)
