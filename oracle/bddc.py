"""BDDC-SO preconditioner, PCG, Lanczos and the adjoint gradient (oracle, FP64).

Definition 1 (abstract multispace BDDC): B r = sum_k Q_k v_k with v_k in V_k
solving a(v_k, z_k) = <r, Q_k z_k> for all z_k in V_k.  Section 3 identifies
BDDC-SO as a = a^Theta, V1 = U_I, Q1 = I and V2 = W-tilde, Q2 = (I - P)E:

  * W = prod W_i, W_i the FE functions on Omega_i vanishing on the Dirichlet
    boundary; a^Theta the sum of subdomain energies.
  * W-tilde = functions of W whose selected coarse DOFs (values at vertices,
    means over (sub)edges and (sub)faces of Theta-hat on Gamma) agree between
    all subdomains sharing the object.
  * P = a^Theta-orthogonal projection onto U_I, so (I - P) keeps the Gamma
    values and replaces the interior by the discrete harmonic extension
    -A_II^{-1} A_IGamma u_Gamma.
  * E = the weighting of eq. (W) or Remark 1.

The V2 problem is solved in two ways.  `apply_definition` states it plainly:
one global constrained (saddle-point) sparse system on W, "a^Theta(v2, z) =
<r, (I-P)E z> for all z in W-tilde", with no coarse space; it is costly and
serves small meshes as the pin of `apply`.  `apply` uses the equivalent
two-level split of W-tilde (Dohrmann 2003, cited in Section 1): the coarse
basis Phi_i of subdomain i solves [A_i C_i^T; C_i 0][Phi_i; Lambda_i] = [0; I]
(energy-minimising functions with unit coarse DOFs), the coarse matrix is
A_c = sum_i R_ci^T Phi_i^T A_i Phi_i R_ci, and the rest of v2 comes from the
constrained local problems [A_i C_i^T; C_i 0][w_i; mu_i] = [r_i; 0].
Sparse LU (SuperLU) and dense Cholesky (LAPACK) are the library primitives
for every solve.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, objects as objmod, partition, weights as wmod


@dataclasses.dataclass
class Subdomain:
    nodes: np.ndarray      # global node ids (non-Dirichlet) in Omega_i-closure, sorted
    A: sp.csr_matrix       # Neumann stiffness on those nodes
    gamma_loc: np.ndarray  # local indices of Gamma nodes
    obj: np.ndarray        # selected global object indices touching Omega_i (sorted)
    C: sp.csr_matrix       # (len(obj), len(nodes)) averaging functionals
    delta: np.ndarray      # weight on each local Gamma node (same order as gamma_loc)


class BDDCSO:
    """The BDDC-SO preconditioner for the Dirichlet Q1 problem on a box mesh."""

    def __init__(self, nx, ny, nz, h, alpha, sub, piece, selection="vef", weighting="card"):
        self.nx, self.ny, self.nz, self.h = nx, ny, nz, h
        self.alpha = np.asarray(alpha, dtype=np.float64)
        self.sub, self.piece = sub, piece
        self.nn = (nx + 1) * (ny + 1) * (nz + 1)
        self.bnd = fem.boundary_node_mask(nx, ny, nz)
        self.A_full = fem.assemble(nx, ny, nz, h, self.alpha).tocsr()
        self.objs = objmod.classify(nx, ny, nz, sub, piece)
        self.sel = objmod.select(self.objs, selection)
        self.n_coarse = len(self.sel)
        parent = wmod.piece_parent(sub, piece)
        pw = wmod.piece_alpha(self.alpha, piece) if weighting == "rho" else None
        self.gamma = self.objs.gamma
        on_gamma = np.zeros(self.nn, dtype=bool)
        on_gamma[self.gamma] = True
        self.on_gamma = on_gamma
        self.interior = np.flatnonzero(~on_gamma & ~self.bnd)

        # subdomains ------------------------------------------------------
        en = fem.element_nodes(nx, ny, nz)
        nsub = int(sub.max()) + 1
        obj_of_sub: Dict[int, List[int]] = {i: [] for i in range(nsub)}
        for o in self.sel:
            for i in self.objs.subdomains[o]:
                obj_of_sub[int(i)].append(int(o))
        self.subs: List[Subdomain] = []
        for i in range(nsub):
            elems = np.flatnonzero(sub == i)
            nodes = np.unique(en[elems])
            nodes = nodes[~self.bnd[nodes]]
            Ai = fem.assemble(nx, ny, nz, h, self.alpha, elems)[nodes][:, nodes].tocsr()
            gl = np.flatnonzero(on_gamma[nodes])
            oi = np.array(sorted(obj_of_sub[i]), dtype=np.int64)
            pos = {int(g): k for k, g in enumerate(nodes)}
            rows, cols, vals = [], [], []
            for r, o in enumerate(oi):
                on = self.objs.nodes[o]
                rows += [r] * len(on)
                cols += [pos[int(v)] for v in on]
                vals += [1.0 / len(on)] * len(on)
            C = sp.csr_matrix((vals, (rows, cols)), shape=(len(oi), len(nodes)))
            d = wmod.delta_all(nodes[gl], i, self.objs.node_pieces, parent, pw)
            self.subs.append(Subdomain(nodes, Ai, gl, oi, C, d))

        # V1 = U_I: the interior nodes of different subdomains do not couple,
        # so A_II is block diagonal; one sparse LU per subdomain.
        self.A_IG = self.A_full[self.interior][:, self.gamma].tocsr()
        self._int_loc, self._int_lu = [], []
        for s in self.subs:
            il = np.flatnonzero(~on_gamma[s.nodes])
            self._int_loc.append(il)
            self._int_lu.append(spla.splu(s.A[il][:, il].tocsc()) if len(il) else None)
        self._gpos = np.full(self.nn, -1, dtype=np.int64)
        self._gpos[self.gamma] = np.arange(len(self.gamma))
        self._obj_index = {int(o): k for k, o in enumerate(self.sel)}
        self._two_level = None
        self._definition = None

    # ------------------------------------------------------------------
    def solve_interior(self, rhs_full: np.ndarray) -> np.ndarray:
        """A_II^{-1} applied to the interior part of a grid vector (0 elsewhere)."""
        out = np.zeros(self.nn)
        for s, il, lu in zip(self.subs, self._int_loc, self._int_lu):
            if lu is not None:
                out[s.nodes[il]] = lu.solve(rhs_full[s.nodes[il]])
        return out

    def harmonic_extension(self, u_gamma: np.ndarray) -> np.ndarray:
        """(I - P) applied to a function given by its Gamma values: keeps them and
        sets the interior to -A_II^{-1} A_IGamma u_Gamma."""
        z = np.zeros(self.nn)
        z[self.gamma] = u_gamma
        t = np.zeros(self.nn)
        t[self.interior] = self.A_IG @ u_gamma
        return z - self.solve_interior(t)

    def _v2_rhs_local(self, r: np.ndarray):
        """v1 = A_II^{-1} r_I and, per subdomain, the right-hand side of the V2
        problem E^T ((I-P)^T r) = delta_i * (r - A v1) on the local Gamma nodes."""
        r = np.where(self.bnd, 0.0, r)
        v1 = self.solve_interior(r)
        res = r - self.A_full @ v1
        loc = []
        for s in self.subs:
            ri = np.zeros(len(s.nodes))
            ri[s.gamma_loc] = s.delta * res[s.nodes[s.gamma_loc]]
            loc.append(ri)
        return v1, loc

    def _finish(self, v1: np.ndarray, w_local) -> np.ndarray:
        """z = v1 + (I - P) E v2 from the local pieces v2_i of v2 in W-tilde."""
        ug = np.zeros(self.nn)
        for s, wi in zip(self.subs, w_local):
            np.add.at(ug, s.nodes[s.gamma_loc], s.delta * wi[s.gamma_loc])
        return v1 + self.harmonic_extension(ug[self.gamma])

    # ------------------------------------------------------------------
    def apply_definition(self, r: np.ndarray) -> np.ndarray:
        """B r with the V2 problem "a^Theta(v2, z) = <r, (I-P)E z> for all z in
        W-tilde" solved as ONE global constrained system on W (continuity of
        the selected coarse DOFs as Lagrange rows).  Direct but costly: used on
        small meshes to pin `apply`."""
        if self._definition is None:
            offs = np.cumsum([0] + [len(s.nodes) for s in self.subs])
            nW = int(offs[-1])
            A_theta = sp.block_diag([s.A for s in self.subs], format="csr")
            grow, gcol, gval = [], [], []
            row = 0
            for o in self.sel:
                ss = [int(i) for i in self.objs.subdomains[o]]

                def crow(i):
                    s = self.subs[i]
                    c = s.C.getrow(int(np.searchsorted(s.obj, o)))
                    return c.indices + offs[i], c.data
                c0, v0 = crow(ss[0])
                for j in ss[1:]:
                    cj, vj = crow(j)
                    grow += [row] * (len(c0) + len(cj))
                    gcol += list(c0) + list(cj)
                    gval += list(v0) + list(-vj)
                    row += 1
            G = sp.csr_matrix((gval, (grow, gcol)), shape=(row, nW))
            K = sp.bmat([[A_theta, G.T], [G, None]], format="csc")
            self._definition = (spla.splu(K).solve, offs, nW, row)
        solve, offs, nW, nrow = self._definition
        v1, loc = self._v2_rhs_local(r)
        w = solve(np.concatenate(loc + [np.zeros(nrow)]))[:nW]
        return self._finish(v1, [w[offs[i]:offs[i + 1]] for i in range(len(self.subs))])

    # ------------------------------------------------------------------
    def coarse_basis(self, i: int):
        """Phi_i, Lambda_i from [A_i C_i^T; C_i 0][Phi; Lambda] = [0; I]."""
        s = self.subs[i]
        nc = s.C.shape[0]
        K = sp.bmat([[s.A, s.C.T], [s.C, None]], format="csc")
        lu = spla.splu(K)
        rhs = np.zeros((len(s.nodes) + nc, nc))
        rhs[len(s.nodes):, :] = np.eye(nc)
        sol = lu.solve(rhs)
        return sol[: len(s.nodes)], sol[len(s.nodes):], lu

    def coarse_dofs(self, i: int) -> np.ndarray:
        """Global coarse-DOF numbers (positions in the selected-object list) of
        the objects of subdomain i, in the order of the rows of C_i."""
        return np.array([self._obj_index[int(o)] for o in self.subs[i].obj], dtype=np.int64)

    def setup_two_level(self):
        """Coarse bases, local constrained-problem factors and the coarse matrix
        A_c = sum_i R_ci^T Phi_i^T A_i Phi_i R_ci with its Cholesky factor."""
        if self._two_level is not None:
            return self._two_level
        bases, lus = [], []
        nc = self.n_coarse
        dense = nc <= 8000
        Ac = np.zeros((nc, nc)) if dense else None
        rows, cols, vals = [], [], []
        for i, s in enumerate(self.subs):
            Phi, _, lu = self.coarse_basis(i)
            bases.append(Phi)
            lus.append(lu)
            Aci = Phi.T @ (s.A @ Phi)
            g = self.coarse_dofs(i)
            if dense:
                Ac[np.ix_(g, g)] += Aci
            else:
                rows.append(np.repeat(g, len(g)))
                cols.append(np.tile(g, len(g)))
                vals.append(Aci.reshape(-1))
        if dense:
            fac = ("chol", np.linalg.cholesky(Ac))
        else:
            Ac = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(nc, nc)).tocsc()
            fac = ("lu", spla.splu(Ac, permc_spec="MMD_AT_PLUS_A"))
        self._two_level = (bases, lus, Ac, fac)
        return self._two_level

    def coarse_solve(self, rc: np.ndarray) -> np.ndarray:
        kind, f = self.setup_two_level()[3]
        return sla.cho_solve((f, True), rc) if kind == "chol" else f.solve(rc)

    def apply(self, r: np.ndarray, coarse=None) -> np.ndarray:
        """z = B r on the full node grid (Dirichlet entries of r ignored, z's 0).

        The V2 solve in its two-level form: v2_i = Phi_i u_c|_i + w_i with
        A_c u_c = sum_i R_ci^T Phi_i^T r_i and w_i from the constrained local
        problem [A_i C_i^T; C_i 0][w_i; mu_i] = [r_i; 0].  coarse: a map
        r_c -> u_c in place of the exact coarse solve (the multilevel
        version, oracle/multilevel.py)."""
        bases, lus, _, _ = self.setup_two_level()
        v1, loc = self._v2_rhs_local(r)
        rc = np.zeros(self.n_coarse)
        for i in range(len(self.subs)):
            np.add.at(rc, self.coarse_dofs(i), bases[i].T @ loc[i])
        uc = coarse(rc) if coarse is not None else self.coarse_solve(rc)
        w = []
        for i, s in enumerate(self.subs):
            nci = s.C.shape[0]
            wi = lus[i].solve(np.concatenate([loc[i], np.zeros(nci)]))[: len(s.nodes)]
            w.append(bases[i] @ uc[self.coarse_dofs(i)] + wi)
        return self._finish(v1, w)

    def coarse_matrix(self):
        bases, _, Ac, _ = self.setup_two_level()
        return Ac, bases

    def operator(self, x: np.ndarray) -> np.ndarray:
        y = self.A_full @ np.where(self.bnd, 0.0, x)
        y[self.bnd] = 0.0
        return y


def build(problem, selection: Optional[str] = None) -> BDDCSO:
    """BDDC-SO for a paper_2001_07289_gb300.inputs.Problem (box partition;
    sub-subdomains from problem.piece when given, else boxes of size L)."""
    sub, piece = partition.box_labels(problem.nx, problem.ny, problem.nz, problem.cuts, problem.L)
    if getattr(problem, "piece", None) is not None:   # sub-subdomains given per element
        piece = np.asarray(problem.piece, dtype=np.int64).reshape(-1)
    return BDDCSO(problem.nx, problem.ny, problem.nz, problem.h, problem.alpha, sub, piece,
                  selection or problem.selection, problem.weights)


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    alphas: np.ndarray
    betas: np.ndarray
    residuals: np.ndarray


def pcg(op, prec, b: np.ndarray, rtol: float, maxit: int = 2000) -> PCGResult:
    """Preconditioned CG from x0 = 0, stopped when ||r_k||_2 <= rtol ||b||_2
    (Section 5: reduce the 2-norm of the residual by the given factor).  The
    iteration count is the number of operator applications."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    res = [nb]
    alphas, betas = [], []
    if nb == 0.0:
        return PCGResult(x, 0, True, np.array([]), np.array([]), np.array(res))
    z = prec(r)
    p = z.copy()
    rz = r @ z
    it = 0
    converged = False
    while it < maxit:
        q = op(p)
        pq = p @ q
        if not pq > 0.0:
            break
        a = rz / pq
        x += a * p
        r -= a * q
        it += 1
        alphas.append(a)
        nr = np.linalg.norm(r)
        res.append(nr)
        if nr <= rtol * nb:
            converged = True
            break
        z = prec(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    return PCGResult(x, it, converged, np.array(alphas), np.array(betas), np.array(res))


def lanczos_extremes(alphas: np.ndarray, betas: np.ndarray):
    """Extreme eigenvalues of the Lanczos matrix T_k of the preconditioned
    operator built from the CG coefficients (Saad, Iterative Methods for Sparse
    Linear Systems, Sec. 6.7.3): T_jj = 1/a_j + b_{j-1}/a_{j-1},
    T_{j,j+1} = sqrt(b_j)/a_j."""
    k = len(alphas)
    if k == 0:
        return np.nan, np.nan
    d = 1.0 / alphas.copy()
    d[1:] += betas[: k - 1] / alphas[: k - 1]
    e = np.sqrt(betas[: k - 1]) / alphas[: k - 1]
    ev = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev[0]), float(ev[-1])


def direct_solve(nx, ny, nz, h, alpha, b: np.ndarray) -> np.ndarray:
    """u = A^{-1} b by sparse LU on the non-Dirichlet nodes (grid layout out)."""
    A, free = fem.dirichlet_system(nx, ny, nz, h, alpha)
    u = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
    u[free] = spla.splu(A).solve(b[free])
    return u


def gradient(nx, ny, nz, h, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dJ/d alpha_e = -lambda_e^T (h K_unit) u_e per element, where A lambda =
    dJ/du: A depends linearly on alpha_e through alpha_e h K_unit (Remark 1)."""
    en = fem.element_nodes(nx, ny, nz)
    K = fem.q1_unit_stiffness()
    ue = u[en]
    le = lam[en]
    return -h * np.einsum("ea,ab,eb->e", le, K, ue)
