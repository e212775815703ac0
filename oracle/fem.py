"""Q1 finite elements on a structured hexahedral mesh (oracle, FP64).

Section 2 (eq. weakform) with the variable coefficient of Remark 1:
a(u, v) = sum_e alpha_e * integral_e grad u . grad v, <F, v> = integral f v,
homogeneous Dirichlet conditions on the whole boundary.  The experiments of
Section 5 use hexahedra, so the FE space is continuous trilinear (Q1).

Mesh: nx*ny*nz cubes of side h; node (i, j, k) has global id
i + (nx+1)*(j + (ny+1)*k); element (i, j, k) has id i + nx*(j + ny*k).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def q1_unit_stiffness() -> np.ndarray:
    """8x8 stiffness of the unit cube: integral of grad phi_a . grad phi_b.

    phi_a = l_ax(x) l_ay(y) l_az(z) with 1-D hats l_0 = 1 - t, l_1 = t, so the
    matrix is the tensor sum k (x) m (x) m + m (x) k (x) m + m (x) m (x) k of the
    1-D stiffness k = [[1, -1], [-1, 1]] and mass m = [[1/3, 1/6], [1/6, 1/3]].
    Local node a = ax + 2*ay + 4*az (x fastest)."""
    k = np.array([[1.0, -1.0], [-1.0, 1.0]])
    m = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
    # np.kron(Z, np.kron(Y, X)) indexes row az*4 + ay*2 + ax
    return (np.kron(m, np.kron(m, k)) + np.kron(m, np.kron(k, m))
            + np.kron(k, np.kron(m, m)))


def q1_stiffness_by_quadrature() -> np.ndarray:
    """The same matrix by a 2x2x2 Gauss rule on the gradients (exact for the
    degree-2-per-axis integrand); an independent route used as a pin."""
    g = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    K = np.zeros((8, 8))
    for qz in g:
        for qy in g:
            for qx in g:
                grads = np.zeros((8, 3))
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    lx = qx if ax else 1 - qx
                    ly = qy if ay else 1 - qy
                    lz = qz if az else 1 - qz
                    dx = 1.0 if ax else -1.0
                    dy = 1.0 if ay else -1.0
                    dz = 1.0 if az else -1.0
                    grads[a] = (dx * ly * lz, lx * dy * lz, lx * ly * dz)
                K += grads @ grads.T / 8.0
    return K


def element_nodes(nx: int, ny: int, nz: int) -> np.ndarray:
    """(n_elems, 8) global node ids of each element, local order ax + 2ay + 4az."""
    idx = np.arange(nx * ny * nz)
    ex, ey, ez = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    px, py = nx + 1, ny + 1
    out = np.empty((nx * ny * nz, 8), dtype=np.int64)
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        out[:, a] = (ex + ax) + px * ((ey + ay) + py * (ez + az))
    return out


def boundary_node_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    """True on nodes of the Dirichlet boundary (whole boundary of the box)."""
    m = np.ones((nz + 1, ny + 1, nx + 1), dtype=bool)
    m[1:nz, 1:ny, 1:nx] = False
    return m.reshape(-1)


def assemble(nx: int, ny: int, nz: int, h: float, alpha: np.ndarray,
             elems: np.ndarray | None = None) -> sp.csr_matrix:
    """Global stiffness on ALL nodes (no boundary condition applied):
    sum over the chosen elements of alpha_e * h * K_unit scattered by node ids.
    The element integral scales as h^(3-2) = h for a cube of side h."""
    en = element_nodes(nx, ny, nz)
    K = q1_unit_stiffness()
    if elems is None:
        elems = np.arange(nx * ny * nz)
    en = en[elems]
    a = alpha[elems] * h
    rows = np.repeat(en, 8, axis=1).reshape(-1)
    cols = np.tile(en, (1, 8)).reshape(-1)
    vals = (a[:, None] * K.reshape(1, 64)).reshape(-1)
    n = (nx + 1) * (ny + 1) * (nz + 1)
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def load_vector(nx: int, ny: int, nz: int, h: float, f) -> np.ndarray:
    """b_n = integral f phi_n by the tensor 2x2x2 Gauss rule per element; the
    rule integrates f * phi_n exactly for f of degree <= 2 per axis times phi."""
    g = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    en = element_nodes(nx, ny, nz)
    ne = nx * ny * nz
    idx = np.arange(ne)
    ex = idx % nx
    ey = (idx // nx) % ny
    ez = idx // (nx * ny)
    b = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
    for qz in g:
        for qy in g:
            for qx in g:
                fv = f((ex + qx) * h, (ey + qy) * h, (ez + qz) * h) * h ** 3 / 8.0
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    w = (qx if ax else 1 - qx) * (qy if ay else 1 - qy) * (qz if az else 1 - qz)
                    np.add.at(b, en[:, a], w * fv)
    b[boundary_node_mask(nx, ny, nz)] = 0.0
    return b


def dirichlet_system(nx, ny, nz, h, alpha):
    """(A_ff, free node ids): the stiffness restricted to non-boundary nodes."""
    A = assemble(nx, ny, nz, h, alpha)
    free = np.flatnonzero(~boundary_node_mask(nx, ny, nz))
    return A[free][:, free].tocsc(), free


def apply_operator_by_elements(nx, ny, nz, h, alpha, x: np.ndarray) -> np.ndarray:
    """The same Dirichlet operator without assembling: y = sum over elements
    of alpha_e h K_unit x_e, done as 64 (a, b) passes over the element grid,
    each adding alpha h K[a, b] times x at the elements' local node b to y at
    their local node a.  For meshes too large to assemble in memory."""
    K = q1_unit_stiffness()
    bnd = boundary_node_mask(nx, ny, nz).reshape(nz + 1, ny + 1, nx + 1)
    xg = np.where(bnd, 0.0, x.reshape(nz + 1, ny + 1, nx + 1))
    ah = alpha.reshape(nz, ny, nx) * h
    y = np.zeros_like(xg)

    def corner(v, a):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        return v[az:az + nz, ay:ay + ny, ax:ax + nx]

    for a in range(8):
        ya = corner(y, a)
        for b in range(8):
            ya += K[a, b] * (ah * corner(xg, b))
    y[bnd] = 0.0
    return y.reshape(-1)


def apply_operator(nx, ny, nz, h, alpha, x: np.ndarray) -> np.ndarray:
    """y = A x on the full node grid, x's boundary entries treated as 0 and y's
    boundary entries set to 0 (the Dirichlet operator in grid layout)."""
    A = assemble(nx, ny, nz, h, alpha)
    bnd = boundary_node_mask(nx, ny, nz)
    xx = np.where(bnd, 0.0, x)
    y = A @ xx
    y[bnd] = 0.0
    return y
