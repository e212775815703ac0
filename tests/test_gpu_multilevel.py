"""Multilevel BDDC-SO on the GPU (options.ml_block = g: the coarse problem
preconditioned by BDDC on blocks of g^3 subdomains, Section 6) against the
oracle's three-level preconditioner (oracle/multilevel.py) on the same
inputs (level-2 weights: cardinality, or stiffness scaling with rho-weights): one application (1e-10 FP64, 2e-5 mixed) and PCG (iterations within
1 / 2 of the oracle's, solution 1e-10 / 1e-8); the level-2 sizes; and one
block holding every subdomain, where the coarse level is the exact coarse
solve and the apply equals the two-level one to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bddc as orc, multilevel as ml  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402

if torch.cuda.is_available():
    from paper_2001_07289_gb300.bddc import BDDC  # noqa: E402

CASES = {
    "uniform": (16, 16, 16, [[4, 8, 12]] * 3, 2, (4, 4, 4), 2, "card"),
    "ragged": (14, 12, 10, [[3, 7, 10], [4, 8], [5]], 2, (4, 3, 2), 2, "card"),
    "rho_L3": (18, 18, 18, [[6, 12]] * 3, 3, (3, 3, 3), 2, "rho"),
}
_cache = {}


def case(name):
    if name not in _cache:
        nx, ny, nz, cuts, L, nsub, g, w = CASES[name]
        a = inputs.alpha_loguniform(nx, ny, nz, -1, 1, 8)
        p = inputs.box_problem(nx, ny, nz, cuts, L, alpha=a, weights=w, rtol=1e-10)
        ref = orc.build(p)
        m2 = ml.CoarseBDDC(ref, nsub, g, "stiffness" if w == "rho" else "card")
        res = orc.pcg(ref.operator, lambda r: ref.apply(r, coarse=m2.apply), p.b, p.rtol)
        _cache[name] = (p, ref, m2, res, g)
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol,dit,atol", [("fp64", 1e-10, 1, 1e-10), ("mixed", 1e-8, 2, 2e-5)])
def test_multilevel_matches_oracle(name, precision, tol, dit, atol):
    p, ref, m2, res, g = case(name)
    pre = BDDC.from_problem(p, precision=precision, ml_block=g)
    info = pre.info()
    assert (info["ml_blocks"], info["ml_coarse2"]) == (m2.nblock, m2.ncc)
    for seed in (3, 4):
        r = inputs.random_node_vector(p.nx, p.ny, p.nz, seed)
        z = pre.apply(torch.from_numpy(r).cuda()).cpu().numpy()
        want = ref.apply(r, coarse=m2.apply)
        assert np.abs(z - want).max() <= atol * np.abs(want).max()
    x, st = pre.solve(torch.from_numpy(p.b).cuda(), p.rtol)
    pre.close()
    assert st["converged"] and res.converged
    assert abs(st["iterations"] - res.iterations) <= dit, (st["iterations"], res.iterations)
    assert np.linalg.norm(x.cpu().numpy() - res.x) <= tol * np.linalg.norm(res.x)


def test_multilevel_graph_pcg_equals_host_loop():
    p, _, _, _, g = case("uniform")
    b = torch.from_numpy(p.b).cuda()
    xs = []
    for graph in (False, True):
        pre = BDDC.from_problem(p, ml_block=g, use_graph=graph)
        x, st = pre.solve(b, p.rtol)
        xs.append((x.cpu().numpy(), st["iterations"]))
        pre.close()
    assert xs[0][1] == xs[1][1] and np.array_equal(xs[0][0], xs[1][0])


def test_one_block_is_the_two_level_preconditioner():
    p = inputs.box_problem(12, 12, 12, [[4, 8]] * 3, 2, alpha=inputs.alpha_loguniform(12, 12, 12, -1, 1, 2))
    r = torch.from_numpy(inputs.random_node_vector(12, 12, 12, 5)).cuda()
    z2 = BDDC.from_problem(p).apply(r).cpu().numpy()
    pre = BDDC.from_problem(p, ml_block=3)
    assert pre.info()["ml_blocks"] == 1 and pre.info()["ml_coarse2"] == 0
    z3 = pre.apply(r).cpu().numpy()
    assert np.abs(z3 - z2).max() <= 1e-11 * np.abs(z2).max()


@pytest.mark.parametrize("sel,piece", [("f", False), ("vef", True), ("f", True)])
def test_multilevel_with_other_sub_partitions(sel, piece):
    """The second level on top of faces-only selections (floating subdomains
    pinned by augmented-Lagrangian terms) and of label-given sub-subdomains
    (synthetic channels, rho-weights, so stiffness-scaled level-2 weights):
    FP64 apply and PCG against the oracle."""
    if piece:
        p = inputs.channels_problem(24, 3, 2, selection=sel, rtol=1e-10)
    else:
        a = inputs.alpha_loguniform(18, 18, 18, -1, 1, 6)
        p = inputs.box_problem(18, 18, 18, [[6, 12]] * 3, 3, alpha=a, selection=sel, rtol=1e-10)
    ref = orc.build(p)
    m2 = ml.CoarseBDDC(ref, (3, 3, 3), 2, "stiffness" if p.weights == "rho" else "card")
    pre = BDDC.from_problem(p, precision="fp64", ml_block=2)
    assert pre.info()["ml_coarse2"] == m2.ncc
    r = inputs.random_node_vector(p.nx, p.ny, p.nz, 3)
    z = pre.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    want = ref.apply(r, coarse=m2.apply)
    assert np.abs(z - want).max() <= 1e-10 * np.abs(want).max()
    x, st = pre.solve(torch.from_numpy(p.b).cuda(), p.rtol)
    pre.close()
    res = orc.pcg(ref.operator, lambda v: ref.apply(v, coarse=m2.apply), p.b, p.rtol)
    assert st["converged"] and abs(st["iterations"] - res.iterations) <= 1
    assert np.linalg.norm(x.cpu().numpy() - res.x) <= 1e-10 * np.linalg.norm(res.x)


@pytest.mark.parametrize("dims,cuts,nsub,g,sub", [
    ((16, 16, 16), [[4, 8, 12]] * 3, (4, 4, 4), 2, 1),        # 2^3 blocks of 2^3 single-subdomain sub-blocks
    ((18, 18, 18), [[3, 6, 9, 12, 15]] * 3, (6, 6, 6), 2, 0),  # 3^3 blocks: a nested-dissection tree at level 2
    ((18, 18, 18), [[3, 6, 9, 12, 15]] * 3, (6, 6, 6), 3, 2),  # ragged sub-blocks (2 + 1 per block and axis)
])
def test_multilevel_subobjects_match_oracle(dims, cuts, nsub, g, sub):
    """Level-2 subobjects (ml_sub = s: level-2 objects split by the sets of
    s^3 sub-blocks sharing them, Section 6) and level-2 coarse problems
    factored by fronts of a nested dissection of the block grid: FP64 apply
    and PCG against the oracle's three-level preconditioner."""
    nx, ny, nz = dims
    a = inputs.alpha_loguniform(nx, ny, nz, -1, 1, 9)
    p = inputs.box_problem(nx, ny, nz, cuts, 2, alpha=a, rtol=1e-10)
    ref = orc.build(p)
    m2 = ml.CoarseBDDC(ref, nsub, g, "card", sub=sub)
    pre = BDDC.from_problem(p, precision="fp64", ml_block=g, ml_sub=sub)
    info = pre.info()
    assert (info["ml_blocks"], info["ml_coarse2"]) == (m2.nblock, m2.ncc)
    r = inputs.random_node_vector(nx, ny, nz, 6)
    z = pre.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    want = ref.apply(r, coarse=m2.apply)
    assert np.abs(z - want).max() <= 1e-10 * np.abs(want).max()
    x, st = pre.solve(torch.from_numpy(p.b).cuda(), p.rtol)
    pre.close()
    res = orc.pcg(ref.operator, lambda v: ref.apply(v, coarse=m2.apply), p.b, p.rtol)
    assert st["converged"] and abs(st["iterations"] - res.iterations) <= 1
    assert np.linalg.norm(x.cpu().numpy() - res.x) <= 1e-10 * np.linalg.norm(res.x)


def test_ml_sub_needs_ml_block():
    p = inputs.box_problem(8, 8, 8, [[4]] * 3, 2)
    with pytest.raises(RuntimeError, match="ml_sub"):
        BDDC.from_problem(p, ml_sub=1)
