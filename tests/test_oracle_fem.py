"""Pins of the oracle's discretisation (Section 2, eq. weakform; Remark 1)."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bddc, fem
from paper_2001_07289_gb300 import inputs


def test_unit_stiffness_matches_quadrature_route():
    K1 = fem.q1_unit_stiffness()
    K2 = fem.q1_stiffness_by_quadrature()
    assert np.abs(K1 - K2).max() < 1e-14


def test_unit_stiffness_closed_form():
    """1/3 on the diagonal, 0 between nodes differing in one coordinate,
    -1/12 between nodes differing in two or three (derived by hand from the
    1-D stiffness/mass tensor sum)."""
    K = fem.q1_unit_stiffness()
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            want = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[d]
            assert abs(K[a, b] - want) < 1e-15
    assert np.abs(K.sum(axis=1)).max() < 1e-15   # constants are in the kernel


def test_assembled_stencil_alpha_one():
    """Interior row of the alpha=1 stiffness: 8h/3 centre, 0 face neighbours,
    -h/6 edge neighbours, -h/12 corners, row sum 0."""
    n = 6
    h = 1.0 / n
    A = fem.assemble(n, n, n, h, np.ones(n ** 3)).tocsr()
    c = 3 + 7 * (3 + 7 * 3)
    row = A.getrow(c).toarray().ravel()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                d = abs(dx) + abs(dy) + abs(dz)
                want = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[d]
                assert abs(row[c + dx + 7 * (dy + 7 * dz)] - want) < 1e-15
    assert abs(row.sum()) < 1e-14


def test_variable_alpha_is_linear_per_element():
    n = 4
    rng = np.random.default_rng(0)
    a = rng.uniform(0.5, 2.0, n ** 3)
    A = fem.assemble(n, n, n, 0.25, a)
    S = sum(a[e] * fem.assemble(n, n, n, 0.25, np.eye(n ** 3)[e]) for e in range(n ** 3))
    assert abs(A - S).max() < 1e-14


def test_rhs_inputs_match_oracle_load_vector():
    n = 6
    h = 1 / n
    b1 = inputs.rhs_constant(n, n, n, h)
    b2 = fem.load_vector(n, n, n, h, lambda x, y, z: np.ones_like(x))
    assert np.abs(b1 - b2).max() < 1e-16
    b3 = inputs.rhs_quadrature(n, n, n, h, inputs.manufactured_f)
    b4 = fem.load_vector(n, n, n, h, inputs.manufactured_f)
    assert np.abs(b3 - b4).max() < 1e-14 * np.abs(b4).max()


def test_manufactured_solution_second_order():
    """Nodal error of the Q1 solution against u = sin(pi x) sin(pi y) sin(pi z)
    falls by ~4 per halving of h (O(h^2))."""
    errs = []
    for n in (8, 16, 32):
        h = 1 / n
        b = fem.load_vector(n, n, n, h, inputs.manufactured_f)
        u = bddc.direct_solve(n, n, n, h, np.ones(n ** 3), b)
        g = np.arange(n + 1) * h
        ue = inputs.manufactured_u(g[None, None, :], g[None, :, None], g[:, None, None]).ravel()
        errs.append(np.abs(u - ue).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs


def test_floating_neumann_kernel():
    """A subdomain matrix that touches no Dirichlet boundary annihilates constants."""
    p = inputs.box_problem(12, 12, 12, [[4, 8]] * 3, 2)
    B = bddc.build(p)
    centre = 1 + 3 * (1 + 3 * 1)
    s = B.subs[centre]
    assert np.abs(s.A @ np.ones(len(s.nodes))).max() < 1e-14
    # and the Dirichlet system is SPD
    A, free = fem.dirichlet_system(12, 12, 12, 1 / 12, np.ones(12 ** 3))
    assert spla.eigsh(A, k=1, which="SA", return_eigenvectors=False)[0] > 0


def test_operator_by_elements_matches_assembled_and_stencil():
    """The element-by-element operator (used where assembly does not fit)
    equals the assembled one on a ragged mesh with variable alpha, and with
    alpha = 1 reproduces the closed-form stencil at an interior node."""
    nx, ny, nz = 7, 5, 6
    h = 1.0 / nx
    a = inputs.alpha_loguniform(nx, ny, nz, -2, 2, 3)
    x = inputs.random_node_vector(nx, ny, nz, 4)
    y1 = fem.apply_operator(nx, ny, nz, h, a, x)
    y2 = fem.apply_operator_by_elements(nx, ny, nz, h, a, x)
    assert np.abs(y1 - y2).max() <= 1e-13 * np.abs(y1).max()
    # unit vector at an interior node: the stencil 8h/3, 0, -h/6, -h/12
    e = np.zeros((nz + 1) * (ny + 1) * (nx + 1))
    i, j, k = 3, 2, 3
    e[i + (nx + 1) * (j + (ny + 1) * k)] = 1.0
    y = fem.apply_operator_by_elements(nx, ny, nz, h, np.ones(nx * ny * nz), e).reshape(nz + 1, ny + 1, nx + 1)
    want = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                d = abs(dx) + abs(dy) + abs(dz)
                assert abs(y[k + dz, j + dy, i + dx] - want[d]) <= 1e-15
