"""Classification of interface DOFs into (sub)objects (oracle).

Section 3: coarse DOFs are values at, or averages over, geometric objects.
BDDC-SO takes its objects from the vertices, edges and faces of the finer
partition Theta-hat that lie on the interface Gamma of Theta.  Classifying a
DOF needs the list of sub-subdomains Omega-hat_j containing it (remark in
Section 3); DOFs with the same list that are connected form one object.

Here:
  * Gamma = non-Dirichlet nodes that belong to two or more subdomains.
  * key(node) = the set of pieces (sub-subdomain labels) of the elements
    around the node.
  * objects = connected components (nodes sharing an element) of Gamma nodes
    with equal keys.
  * type = by the number of sub-subdomains in the key (Section 3: the
    objects are the vertices, edges and faces of Theta-hat, classified from
    the list of sub-subdomains containing each DOF): 2 -> face, 3 or 4 ->
    edge, more -> vertex.  In a tensor-product Theta-hat these are 2, 4 and
    8, whatever the number of nodes of the object (a face between two
    one-node intervals is still a face).  A one-node object is a point value
    whatever its type, so the type only matters for the selection variants.
  * selection (Table 1 / Section 5.2 variants): "vef" keeps every object,
    "ve" vertices and edges, "f" faces only, "v" vertices only.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from . import fem


def node_element_labels(nx: int, ny: int, nz: int, labels: np.ndarray) -> np.ndarray:
    """(n_nodes, 8) labels of the up-to-8 elements around each node, -1 where
    the element lies outside the mesh."""
    pad = np.full((nz + 2, ny + 2, nx + 2), -1, dtype=np.int64)
    pad[1:-1, 1:-1, 1:-1] = labels.reshape(nz, ny, nx)
    out = np.empty(((nx + 1) * (ny + 1) * (nz + 1), 8), dtype=np.int64)
    c = 0
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                out[:, c] = pad[dz:dz + nz + 1, dy:dy + ny + 1, dx:dx + nx + 1].reshape(-1)
                c += 1
    return out


def _sorted_unique_rows(lab: np.ndarray) -> np.ndarray:
    """Each row's distinct non-negative values, sorted, padded with -1 at the end."""
    s = np.sort(lab, axis=1)
    dup = np.zeros_like(s, dtype=bool)
    dup[:, 1:] = s[:, 1:] == s[:, :-1]
    s = np.where(dup, -1, s)
    # push -1 entries to the end while keeping order of the rest
    key = np.where(s < 0, np.iinfo(np.int64).max, s)
    s = np.sort(key, axis=1)
    return np.where(s == np.iinfo(np.int64).max, -1, s)


@dataclasses.dataclass
class Objects:
    nodes: List[np.ndarray]          # global node ids of each object
    kind: np.ndarray                 # 0 vertex, 1 edge, 2 face
    subdomains: List[np.ndarray]     # subdomains containing the object
    key: List[np.ndarray]            # pieces containing the object
    gamma: np.ndarray                # global node ids on Gamma
    node_subs: np.ndarray            # (n_nodes, 8) sorted distinct subdomains per node
    node_pieces: np.ndarray          # (n_nodes, 8) sorted distinct pieces per node

    def __len__(self):
        return len(self.nodes)

    def counts(self):
        return {t: int(np.sum(self.kind == k)) for k, t in enumerate(("vertices", "edges", "faces"))}


def classify(nx: int, ny: int, nz: int, sub: np.ndarray, piece: np.ndarray) -> Objects:
    """All objects of Theta-hat lying on Gamma."""
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    node_subs = _sorted_unique_rows(node_element_labels(nx, ny, nz, sub))
    node_pieces = _sorted_unique_rows(node_element_labels(nx, ny, nz, piece))
    nsub = np.sum(node_subs >= 0, axis=1)
    bnd = fem.boundary_node_mask(nx, ny, nz)
    on_gamma = (nsub >= 2) & ~bnd
    gamma = np.flatnonzero(on_gamma)
    if len(gamma) == 0:                      # one subdomain: no interface, no objects
        return Objects([], np.zeros(0, dtype=np.int64), [], [], gamma, node_subs, node_pieces)
    # key id per Gamma node
    _, key_id = np.unique(node_pieces[gamma], axis=0, return_inverse=True)
    key_full = np.full(nn, -1, dtype=np.int64)
    key_full[gamma] = key_id.reshape(-1)
    # edges between Gamma nodes of equal key sharing an element (26-neighbours)
    grid = key_full.reshape(nz + 1, ny + 1, nx + 1)
    ids = np.arange(nn).reshape(nz + 1, ny + 1, nx + 1)
    rows, cols = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) <= (0, 0, 0):
                    continue
                a = (slice(max(0, -dz), nz + 1 - max(0, dz)),
                     slice(max(0, -dy), ny + 1 - max(0, dy)),
                     slice(max(0, -dx), nx + 1 - max(0, dx)))
                b = (slice(max(0, dz), nz + 1 - max(0, -dz)),
                     slice(max(0, dy), ny + 1 - max(0, -dy)),
                     slice(max(0, dx), nx + 1 - max(0, -dx)))
                ka, kb = grid[a], grid[b]
                m = (ka >= 0) & (ka == kb)
                rows.append(ids[a][m])
                cols.append(ids[b][m])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    g = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(nn, nn)).tocsr()
    g = g[gamma][:, gamma]
    ncomp, comp = connected_components(g, directed=False)
    order = np.argsort(comp, kind="stable")
    splits = np.flatnonzero(np.diff(comp[order])) + 1
    groups = np.split(gamma[order], splits)
    # deterministic object order: by (type, lowest node id)
    kinds = []
    for grp in groups:
        npieces = int(np.sum(node_pieces[grp[0]] >= 0))
        kinds.append(2 if npieces == 2 else (1 if npieces <= 4 else 0))
    kinds = np.array(kinds, dtype=np.int64)
    first = np.array([grp.min() for grp in groups], dtype=np.int64)
    perm = np.lexsort((first, kinds))
    groups = [np.sort(groups[p]) for p in perm]
    kinds = kinds[perm]
    subs = [node_subs[grp[0]][node_subs[grp[0]] >= 0] for grp in groups]
    keys = [node_pieces[grp[0]][node_pieces[grp[0]] >= 0] for grp in groups]
    return Objects(groups, kinds, subs, keys, gamma, node_subs, node_pieces)


def select(objs: Objects, selection: str = "vef") -> np.ndarray:
    """Indices of the objects carrying a coarse DOF."""
    allowed = {"vef": (0, 1, 2), "ve": (0, 1), "vf": (0, 2), "f": (2,), "v": (0,), "ef": (1, 2)}[selection]
    return np.flatnonzero(np.isin(objs.kind, allowed))
