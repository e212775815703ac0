"""Acceptable-path check of a constraint selection (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The remark after Theorem 1: the bound of Theorem 1 uses the standard BDDC
result for the auxiliary BDDC-A on Theta-hat, which needs enough primal
constraints that every pair of neighbouring sub-subdomains is joined by an
acceptable path; all edge or all face subobjects on the original interface
Gamma guarantee that.  The paper cites the definition; the reading used here
(with the coefficient condition of the multi-material setting it cites):

  * a pair: two sub-subdomains of different subdomains whose closures share a
    node off the Dirichlet boundary;
  * direct: the pair shares a selected edge or face object (both lie in the
    object's key, the set of sub-subdomains containing it), or every free
    node the two share lies in a selected object (the contact is primal);
  * links of a path: two sub-subdomains of one subdomain sharing an element
    face (functions of W-tilde are continuous inside a subdomain), or two of
    different subdomains sharing an element face and either a selected face
    object or only primal free nodes;
  * quality of a path from i to j: min(1, min of rho over the path /
    min(rho_i, rho_j)), rho of a sub-subdomain = the mean of alpha over its
    elements; a pair takes the best quality over its paths.

Written as plain definitions: the best quality of a pair is the largest
threshold t among the rho values such that i and j are connected through
sub-subdomains with rho >= t, found by recomputing the connected components
for every threshold.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from . import fem, objects as objmod


def _face_contacts(nx, ny, nz, lab):
    """Pairs (a, b), a < b, of labels of elements sharing an element face."""
    g = lab.reshape(nz, ny, nx)
    out = set()
    for ax in range(3):
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[2 - ax] = slice(0, -1)
        sl_b[2 - ax] = slice(1, None)
        a, b = g[tuple(sl_a)].reshape(-1), g[tuple(sl_b)].reshape(-1)
        m = a != b
        for u, v in zip(np.minimum(a[m], b[m]), np.maximum(a[m], b[m])):
            out.add((int(u), int(v)))
    return out


def acceptable_paths(nx, ny, nz, sub, piece, alpha, selection="vef"):
    """Pairs, direct pairs, pairs without an acceptable path and the smallest
    best-path quality; also the per-pair qualities {(i, j): q} (None: no path)."""
    objs = objmod.classify(nx, ny, nz, sub, piece)
    sel = set(int(k) for k in objmod.select(objs, selection))
    npiece = int(piece.max()) + 1
    piece_sub = np.zeros(npiece, dtype=np.int64)
    piece_sub[piece] = sub
    alpha = np.ones(nx * ny * nz) if alpha is None else np.asarray(alpha, dtype=np.float64).reshape(-1)
    rho = np.bincount(piece, weights=alpha, minlength=npiece) / np.bincount(piece, minlength=npiece)
    # pairs: pieces of different subdomains around one free node; a pair's
    # contact is primal while each such node lies in a selected object
    bnd = fem.boundary_node_mask(nx, ny, nz)
    primal_node = np.zeros(len(bnd), dtype=bool)
    for o in sel:
        primal_node[objs.nodes[o]] = True
    pairs, open_contact = set(), set()
    for node in np.flatnonzero(~bnd):
        row = objs.node_pieces[node]
        ps = row[row >= 0]
        for x in range(len(ps)):
            for y in range(x + 1, len(ps)):
                if piece_sub[ps[x]] != piece_sub[ps[y]]:
                    pairs.add((int(ps[x]), int(ps[y])))
                    if not primal_node[node]:
                        open_contact.add((int(ps[x]), int(ps[y])))
    direct = set(p for p in pairs if p not in open_contact)
    links = set()
    for o in sel:
        key = [int(k) for k in objs.key[o]]
        if objs.kind[o] == 0:
            continue
        for x in range(len(key)):
            for y in range(x + 1, len(key)):
                direct.add((min(key[x], key[y]), max(key[x], key[y])))
        if objs.kind[o] == 2:
            links.add((min(key), max(key)))
    for u, v in _face_contacts(nx, ny, nz, piece):
        if piece_sub[u] == piece_sub[v] or (u, v) not in open_contact:
            links.add((u, v))
    # best path quality by thresholds
    L = np.array(sorted(links), dtype=np.int64).reshape(-1, 2)
    todo = sorted(p for p in pairs if p not in direct)
    best = {p: None for p in todo}
    for t in sorted(set(rho.tolist()), reverse=True):
        keep = rho >= t
        m = keep[L[:, 0]] & keep[L[:, 1]]
        g = sp.coo_matrix((np.ones(int(m.sum())), (L[m, 0], L[m, 1])), shape=(npiece, npiece))
        _, comp = connected_components(g, directed=False)
        for (i, j) in todo:
            if best[(i, j)] is None and keep[i] and keep[j] and comp[i] == comp[j]:
                best[(i, j)] = min(1.0, t / min(rho[i], rho[j]))
    q = [v for v in best.values() if v is not None]
    return {"n_pieces": npiece, "n_pairs": len(pairs), "n_direct": len(pairs & direct),
            "n_without_path": sum(v is None for v in best.values()),
            "min_ratio": min(q) if q else 1.0, "quality": best}
