"""Pins of the oracle's second level (multilevel BDDC-SO, Section 6): BDDC on
the coarse problem A_c with blocks of subdomains.

- the two-level form (level-2 basis Psi, exact level-2 coarse solve) equals
  Definition 1 solved as one global constrained system on the blocks;
- M2 is a BDDC preconditioner of A_c: symmetric, lambda_min(M2 A_c) >= 1
  (the multispace bound behind Theorem 1, now on the coarse level), with
  cardinality and with stiffness-scaled weights (each a partition of unity:
  the bound needs only that);
- one block holding every subdomain: no coarse interface, M2 = A_c^{-1}, so
  the three-level preconditioner is the two-level one;
- the three-level preconditioner B3 is symmetric with lambda_min(B3 A) >= 1,
  and PCG with it reaches the two-level solution.
"""
import numpy as np
import pytest

from oracle import bddc as orc, multilevel as ml
from paper_2001_07289_gb300 import inputs

CASES = {
    "uniform": (16, 16, 16, [[4, 8, 12]] * 3, 2, (4, 4, 4), 2),
    "ragged": (14, 12, 10, [[3, 7, 10], [4, 8], [5]], 2, (4, 3, 2), 2),
    "rho": (12, 12, 12, [[3, 6, 9]] * 3, 3, (4, 4, 4), 2),
}


def build(name):
    nx, ny, nz, cuts, L, nsub, g = CASES[name]
    a = inputs.alpha_loguniform(nx, ny, nz, -1, 1, 4)
    rho = name == "rho"
    p = inputs.box_problem(nx, ny, nz, cuts, L, alpha=a, weights="rho" if rho else "card")
    ref = orc.build(p)
    return p, ref, ml.CoarseBDDC(ref, nsub, g, "stiffness" if rho else "card")


@pytest.mark.parametrize("name", list(CASES))
def test_two_level_form_equals_definition(name):
    _, ref, m2 = build(name)
    assert m2.ncc > 0 and m2.nblock > 1
    rng = np.random.default_rng(2)
    for _ in range(2):
        r = rng.standard_normal(ref.n_coarse)
        a, b = m2.apply(r), m2.apply_definition(r)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("name", ["uniform", "ragged", "rho"])
def test_coarse_level_is_bddc(name):
    _, ref, m2 = build(name)
    M = np.array([m2.apply(e) for e in np.eye(ref.n_coarse)]).T
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    ev = np.linalg.eigvals(M @ m2.Ac).real
    assert ev.min() >= 1 - 1e-10
    assert ev.max() > 1 + 1e-3       # a real preconditioner, not the inverse


def test_one_block_is_the_exact_coarse_solve():
    p = inputs.box_problem(12, 12, 12, [[4, 8]] * 3, 2)
    ref = orc.build(p)
    m2 = ml.CoarseBDDC(ref, (3, 3, 3), 3)
    assert m2.nblock == 1 and m2.ncc == 0
    r = np.random.default_rng(3).standard_normal(ref.n_coarse)
    want = ref.coarse_solve(r)
    assert np.abs(m2.apply(r) - want).max() <= 1e-12 * np.abs(want).max()


def test_three_level_spectrum_and_pcg():
    a = inputs.alpha_loguniform(9, 9, 9, -1, 1, 5)
    p = inputs.box_problem(9, 9, 9, [[3, 6]] * 3, 2, alpha=a)
    ref = orc.build(p)
    m2 = ml.CoarseBDDC(ref, (3, 3, 3), 2)
    free = np.flatnonzero(~ref.bnd)
    e = np.zeros(ref.nn)
    cols = []
    for q in free:
        e[:] = 0.0
        e[q] = 1.0
        cols.append(ref.apply(e, coarse=m2.apply)[free])
    B = np.array(cols).T
    A = ref.A_full[free][:, free].toarray()
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    ev = np.linalg.eigvals(B @ A).real
    assert ev.min() >= 1 - 1e-10 and ev.max() > 1.01
    r2 = orc.pcg(ref.operator, ref.apply, p.b, 1e-10)
    r3 = orc.pcg(ref.operator, lambda r: ref.apply(r, coarse=m2.apply), p.b, 1e-10)
    assert r3.converged and r3.iterations >= r2.iterations
    assert np.linalg.norm(r3.x - r2.x) <= 1e-9 * np.linalg.norm(r2.x)


def test_weights_partition_of_unity():
    for name, kind in (("ragged", "card"), ("rho", "stiffness")):
        _, ref, m2 = build(name)
        tot = np.zeros(ref.n_coarse)
        for d, w in zip(m2.bdofs, m2.wb):
            np.add.at(tot, d, w)
        assert np.abs(tot - 1).max() < 1e-13


@pytest.mark.parametrize("name", ["rho"])
def test_level2_subobjects(name):
    """Sub-blocks of one subdomain inside the blocks (subobjects on the coarse
    level, Section 6): the two forms still agree, lambda_min(M2 A_c) >= 1, and
    since every block-level constraint is implied by the finer ones W-tilde_2
    shrinks, so lambda_max (the largest value of the BDDC Rayleigh quotient
    over W-tilde_2) cannot grow."""
    nx, ny, nz, cuts, L, nsub, g = CASES[name]
    a = inputs.alpha_loguniform(nx, ny, nz, -1, 1, 4)
    p = inputs.box_problem(nx, ny, nz, cuts, L, alpha=a)
    ref = orc.build(p)
    ev = {}
    for sub in (0, 1):
        m2 = ml.CoarseBDDC(ref, nsub, g, "card", sub)
        r = np.random.default_rng(4).standard_normal(ref.n_coarse)
        x, y = m2.apply(r), m2.apply_definition(r)
        assert np.abs(x - y).max() <= 1e-12 * np.abs(x).max()
        M = np.array([m2.apply(e) for e in np.eye(ref.n_coarse)]).T
        e = np.linalg.eigvals(M @ m2.Ac).real
        assert e.min() >= 1 - 1e-10
        ev[sub] = (m2.ncc, e.max())
    assert ev[1][0] > ev[0][0] and ev[1][1] <= ev[0][1] * (1 + 1e-10)
