"""Multilevel BDDC-SO: the second level (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 6 (Conclusion) names the multilevel version as the way to use
BDDC-SO beyond the coarse-problem size that a direct solve allows: the
coarse problem A_c u_c = r_c is not solved exactly but preconditioned by one
application of BDDC on the coarse level (three-level BDDC).  The paper gives
no formulas for it; the reading used here applies Definition 1 once more,
with the coarse problem in the place of the fine one:

  * coarse "elements": the subdomains, with the local coarse matrices
    A_c^(i) = Phi_i^T A_i Phi_i on their coarse DOFs;
  * coarse "subdomains": blocks of g x g x g subdomains of the box grid (the
    last block of an axis takes what is left);
  * coarse interface Gamma_2: the coarse DOFs shared by two or more blocks;
    V1 = the block-interior coarse DOFs (block-diagonal A_c,II);
  * level-2 objects: the Gamma_2 DOFs grouped by the set of blocks sharing
    them (for box blocks each such set is connected), typed by its size (2
    face, 3 or 4 edge, more vertex), all selected, each constraint the mean
    of the object's coarse DOF values (a one-DOF object: its value);
    with sub-blocks of s x s x s subdomains inside every block (BDDC-SO on
    the coarse level: Section 6 points at the freedom to define subobjects
    on every coarser level), the Gamma_2 DOFs are grouped by the set of
    sub-blocks sharing them instead;
  * weights: 1 / (number of blocks sharing the DOF) (eq. (W) with blocks),
    or, with Remark 1's rho-weights on the first level, stiffness scaling
    on the second, the coarse-level analogue of Remark 1 (the coarse level
    has no coefficient of its own): delta_k(j) = (A_k)_jj / sum over the
    blocks k' sharing j of (A_k')_jj;
  * the level-2 coarse problem (one DOF per level-2 object) solved exactly.

M2 is then a BDDC preconditioner of A_c and the three-level preconditioner
is the two-level one with u_c = M2 r_c instead of A_c^{-1} r_c.  M2 is
written twice, like the first level: `apply` in its two-level form (level-2
coarse basis Psi from the block saddle-point problems, exact level-2 coarse
solve, constrained block problems) and `apply_definition` (the W-tilde_2
problem as one global constrained system); the tests pin them equal.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np
import scipy.linalg as sla


class CoarseBDDC:
    def __init__(self, ref, nsub: Sequence[int], g: int, weights: str = "card", sub: int = 0):
        """ref: an oracle BDDCSO; nsub: subdomains per axis; g: block width in
        subdomains; weights: "card" or "stiffness" (see the module text); sub:
        sub-block width in subdomains for level-2 subobjects (0: none)."""
        bases, _, Ac, _ = ref.setup_two_level()
        self.Ac = np.asarray(Ac.todense()) if hasattr(Ac, "todense") else np.asarray(Ac)
        nc = ref.n_coarse
        self.nc = nc
        nsx, nsy, nsz = nsub
        nbx, nby, nbz = (-(-nsx // g), -(-nsy // g), -(-nsz // g))
        self.nblock = nbx * nby * nbz
        block_of_sub, part_of_sub = [], []
        for i in range(nsx * nsy * nsz):
            sx, sy, sz = i % nsx, (i // nsx) % nsy, i // (nsx * nsy)
            b = sx // g + nbx * (sy // g + nby * (sz // g))
            block_of_sub.append(b)
            if sub:   # sub-block inside the block: local coordinates // sub
                part_of_sub.append((b, (sx % g) // sub, (sy % g) // sub, (sz % g) // sub))
            else:
                part_of_sub.append((b,))
        # local coarse matrices and the blocks sharing each coarse DOF
        blocks_of: List[set] = [set() for _ in range(nc)]
        parts_of: List[set] = [set() for _ in range(nc)]
        self.sub_dofs, self.sub_Ac = [], []
        for i, s in enumerate(ref.subs):
            gi = ref.coarse_dofs(i)
            self.sub_dofs.append(gi)
            self.sub_Ac.append(bases[i].T @ (s.A @ bases[i]))
            for j in gi:
                blocks_of[int(j)].add(block_of_sub[i])
                parts_of[int(j)].add(part_of_sub[i])
        self.bset = [frozenset(b) for b in blocks_of]
        # block DOF sets (sorted) and assembled block matrices
        self.bdofs: List[np.ndarray] = []
        self.Ab: List[np.ndarray] = []
        for k in range(self.nblock):
            d = np.array(sorted(j for j in range(nc) if k in self.bset[j]), dtype=np.int64)
            pos = {int(j): q for q, j in enumerate(d)}
            A = np.zeros((len(d), len(d)))
            for i in range(len(ref.subs)):
                if block_of_sub[i] == k:
                    li = [pos[int(j)] for j in self.sub_dofs[i]]
                    A[np.ix_(li, li)] += self.sub_Ac[i]
            self.bdofs.append(d)
            self.Ab.append(A)
        self.gamma2 = np.array([len(b) >= 2 for b in self.bset])
        # weights per block on its own DOFs
        if weights == "card":
            self.wb = [np.array([1.0 / len(self.bset[int(j)]) for j in d]) for d in self.bdofs]
        elif weights == "stiffness":
            dsum = np.zeros(nc)
            for d, A in zip(self.bdofs, self.Ab):
                np.add.at(dsum, d, np.diag(A))
            self.wb = [np.diag(A) / dsum[d] for d, A in zip(self.bdofs, self.Ab)]
        else:
            raise ValueError(weights)
        # level-2 objects: Gamma_2 DOFs grouped by their block set
        groups: Dict[frozenset, List[int]] = {}
        for j in range(nc):
            if self.gamma2[j]:
                groups.setdefault(frozenset(parts_of[j]), []).append(j)
        self.objs = [np.array(v, dtype=np.int64) for v in sorted(groups.values(), key=lambda v: v[0])]
        self.obj_blocks = [self.bset[int(o[0])] for o in self.objs]
        self.kind = np.array([2 if len(b) == 2 else (1 if len(b) <= 4 else 0) for b in self.obj_blocks])
        self.ncc = len(self.objs)
        # block constraint rows, saddle-point bases, level-2 coarse matrix
        self.bobj, self.C, self.Psi, self.K = [], [], [], []
        Acc = np.zeros((self.ncc, self.ncc))
        for k in range(self.nblock):
            d = self.bdofs[k]
            pos = {int(j): q for q, j in enumerate(d)}
            oo = [q for q, b in enumerate(self.obj_blocks) if k in b]
            C = np.zeros((len(oo), len(d)))
            for r, q in enumerate(oo):
                for j in self.objs[q]:
                    C[r, pos[int(j)]] = 1.0 / len(self.objs[q])
            n, m = len(d), len(oo)
            K = np.block([[self.Ab[k], C.T], [C, np.zeros((m, m))]])
            rhs = np.zeros((n + m, m))
            rhs[n:, :] = np.eye(m)
            Psi = np.linalg.solve(K, rhs)[:n] if m else np.zeros((n, 0))
            self.bobj.append(np.array(oo, dtype=np.int64))
            self.C.append(C)
            self.Psi.append(Psi)
            self.K.append(K)
            if m:
                Acc[np.ix_(oo, oo)] += Psi.T @ self.Ab[k] @ Psi
        self.Acc = Acc
        self.Acc_chol = np.linalg.cholesky(Acc) if self.ncc else None
        # interior solves
        self.bint = [np.flatnonzero(~self.gamma2[d]) for d in self.bdofs]

    # ------------------------------------------------------------------
    def _interior(self, r: np.ndarray) -> np.ndarray:
        """A_c,II^{-1} r_I (block-diagonal), zero on Gamma_2."""
        u = np.zeros(self.nc)
        for k, d in enumerate(self.bdofs):
            il = self.bint[k]
            if len(il):
                u[d[il]] = np.linalg.solve(self.Ab[k][np.ix_(il, il)], r[d[il]])
        return u

    def _finish(self, uI: np.ndarray, v_blocks) -> np.ndarray:
        """u_I + (I - P_2) E_2 v: weighted average of the blocks' Gamma_2
        values, then the harmonic extension into the block interiors."""
        vg = np.zeros(self.nc)
        for k, d in enumerate(self.bdofs):
            gl = self.gamma2[d]
            np.add.at(vg, d[gl], self.wb[k][gl] * v_blocks[k][gl])
        t = self.Ac @ vg
        t[self.gamma2] = 0.0
        return uI + vg - self._interior(t)

    def _local_rhs(self, r: np.ndarray):
        uI = self._interior(r)
        res = r - self.Ac @ uI
        loc = []
        for k, d in enumerate(self.bdofs):
            rk = np.where(self.gamma2[d], self.wb[k] * res[d], 0.0)
            loc.append(rk)
        return uI, loc

    def apply(self, r: np.ndarray) -> np.ndarray:
        """M2 r, two-level form of Definition 1 on the coarse level."""
        uI, loc = self._local_rhs(r)
        rcc = np.zeros(self.ncc)
        for k in range(self.nblock):
            if len(self.bobj[k]):
                rcc[self.bobj[k]] += self.Psi[k].T @ loc[k]
        ucc = sla.cho_solve((self.Acc_chol, True), rcc) if self.ncc else rcc
        v = []
        for k in range(self.nblock):
            n, m = len(self.bdofs[k]), len(self.bobj[k])
            w = np.linalg.solve(self.K[k], np.concatenate([loc[k], np.zeros(m)]))[:n]
            v.append(self.Psi[k] @ ucc[self.bobj[k]] + w)
        return self._finish(uI, v)

    def apply_definition(self, r: np.ndarray) -> np.ndarray:
        """M2 r with the W-tilde_2 problem solved as one constrained system on
        the product of the block spaces (continuity of every level-2 object's
        mean as Lagrange rows between the blocks sharing it)."""
        uI, loc = self._local_rhs(r)
        offs = np.cumsum([0] + [len(d) for d in self.bdofs])
        nW = int(offs[-1])
        A = sla.block_diag(*self.Ab)
        rows = []
        for q, blocks in enumerate(self.obj_blocks):
            bl = sorted(blocks)

            def row(k):
                z = np.zeros(nW)
                r_ = list(self.bobj[k]).index(q)
                z[offs[k]:offs[k + 1]] = self.C[k][r_]
                return z
            r0 = row(bl[0])
            for k in bl[1:]:
                rows.append(r0 - row(k))
        G = np.array(rows).reshape(-1, nW)
        K = np.block([[A, G.T], [G, np.zeros((len(G), len(G)))]])
        w = np.linalg.solve(K, np.concatenate(loc + [np.zeros(len(G))]))[:nW]
        return self._finish(uI, [w[offs[k]:offs[k + 1]] for k in range(self.nblock)])
