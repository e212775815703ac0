"""Constraint-selection variants (Section 5: BDDC-SO with vertices and
edges, vertices and faces, or vertices only) on the GPU against the oracle
built with the same selection: apply, PCG iterations and solution, for the
FP64 and mixed paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bddc as orc  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402

_cache = {}


def _case(sel):
    if sel not in _cache:
        a = inputs.alpha_loguniform(14, 11, 9, -1, 1, 1)
        p = inputs.box_problem(14, 11, 9, [[5, 9], [4], [3, 6]], 3, alpha=a, selection=sel)
        _cache[sel] = (p, orc.build(p))
    return _cache[sel]


@pytest.mark.parametrize("sel", ["ve", "vf", "v"])
@pytest.mark.parametrize("precision,tol,dit", [("fp64", 1e-10, 1), ("mixed", 1e-8, 2)])
def test_selection_matches_oracle(sel, precision, tol, dit):
    from paper_2001_07289_gb300.bddc import BDDC
    p, ref = _case(sel)
    pre = BDDC.from_problem(p, precision=precision)
    assert pre.info()["n_coarse"] == len(ref.sel)
    r = inputs.random_node_vector(p.nx, p.ny, p.nz, 3)
    z = pre.apply(torch.from_numpy(r).cuda()).cpu().numpy()
    zr = ref.apply(r)
    atol = 1e-10 if precision == "fp64" else 2e-5
    assert np.abs(z - zr).max() <= atol * np.abs(zr).max()
    b = inputs.random_node_vector(p.nx, p.ny, p.nz, 4)
    x, st = pre.solve(torch.from_numpy(b).cuda(), 1e-10)
    res = orc.pcg(ref.operator, ref.apply, b, 1e-10)
    assert st["converged"] and res.converged
    assert abs(st["iterations"] - res.iterations) <= dit, (st["iterations"], res.iterations)
    assert np.linalg.norm(x.cpu().numpy() - res.x) <= tol * np.linalg.norm(res.x)
    pre.close()


def test_fewer_constraints_more_iterations():
    """Dropping constraints enlarges W-tilde: v needs at least as many PCG
    iterations as ve and vf, which need at least as many as vef."""
    from paper_2001_07289_gb300.bddc import BDDC
    it = {}
    for sel in ("vef", "ve", "vf", "v"):
        p = inputs.box_problem(24, 24, 24, [[8, 16]] * 3, 4, selection=sel)
        pre = BDDC.from_problem(p)
        _, st = pre.solve(torch.from_numpy(inputs.random_node_vector(24, 24, 24, 9)).cuda(), 1e-8)
        it[sel] = st["iterations"]
        pre.close()
    assert it["vef"] <= min(it["ve"], it["vf"]) and max(it["ve"], it["vf"]) <= it["v"], it
