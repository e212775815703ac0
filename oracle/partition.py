"""The partition Theta and the sub-partition Theta-hat (oracle).

Section 3: Theta = {Omega_i} is a non-overlapping partition of the mesh into
connected unions of elements (here boxes cut by per-axis planes, as in the
experiments of Section 5).  Theta-hat = {Omega-hat_j} splits every Omega_i
further into sub-subdomains of characteristic size L; the split is decided
locally per subdomain (remark in Section 3).  The paper leaves the rule open;
the reading used here: a subdomain side of w elements is cut into
s = ceil(w / L) pieces with boundaries at floor(k w / s), k = 1 .. s-1, so
every piece is at most L wide and pieces nest when L divides w.

Both partitions are returned as per-element labels so that non-tensor
sub-partitions (such as the L-shaped piece of Figure 1) can be expressed too.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np


def slab_bounds(n: int, cuts: Sequence[int]) -> List[Tuple[int, int]]:
    """[(lo, hi)] element ranges of the slabs between consecutive cut planes."""
    b = [0] + list(cuts) + [n]
    for a, c in zip(b[:-1], b[1:]):
        if not a < c:
            raise ValueError("cut planes must be strictly increasing inside (0, n)")
    return list(zip(b[:-1], b[1:]))


def subdivide(lo: int, hi: int, L: int) -> List[int]:
    """Interior boundaries of the pieces of the slab [lo, hi): s = ceil(w/L)
    pieces with boundaries lo + floor(k w / s)."""
    if L < 1:
        raise ValueError("L must be >= 1")
    w = hi - lo
    s = max(1, math.ceil(w / L))
    return [lo + (k * w) // s for k in range(1, s)]


def axis_labels(n: int, cuts: Sequence[int], L: int) -> Tuple[np.ndarray, np.ndarray, List[int]]:
    """Per-element slab index and piece index along one axis, and the list of
    all piece boundaries (Theta cuts and Theta-hat-only cuts, sorted)."""
    slab = np.zeros(n, dtype=np.int64)
    piece = np.zeros(n, dtype=np.int64)
    hat_cuts: List[int] = []
    p = 0
    for s, (lo, hi) in enumerate(slab_bounds(n, cuts)):
        slab[lo:hi] = s
        inner = subdivide(lo, hi, L)
        bounds = [lo] + inner + [hi]
        for a, c in zip(bounds[:-1], bounds[1:]):
            piece[a:c] = p
            p += 1
        hat_cuts += inner
        if hi < n:
            hat_cuts.append(hi)
    return slab, piece, sorted(hat_cuts)


def box_labels(nx: int, ny: int, nz: int, cuts: Sequence[Sequence[int]], L: int):
    """Per-element subdomain label and sub-subdomain (piece) label for the box
    partition given by per-axis cuts and the subdivision rule.  Labels are
    numbered x fastest."""
    sx, px_, _ = axis_labels(nx, cuts[0], L)
    sy, py_, _ = axis_labels(ny, cuts[1], L)
    sz, pz_, _ = axis_labels(nz, cuts[2], L)
    nsx, nsy = sx.max() + 1, sy.max() + 1
    npx, npy = px_.max() + 1, py_.max() + 1
    sub = (sx[None, None, :] + nsx * (sy[None, :, None] + nsy * sz[:, None, None]))
    pc = (px_[None, None, :] + npx * (py_[None, :, None] + npy * pz_[:, None, None]))
    return sub.reshape(-1).astype(np.int64), pc.reshape(-1).astype(np.int64)
