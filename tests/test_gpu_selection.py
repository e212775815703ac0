"""Constraint-selection variants (Section 5: BDDC-SO with vertices and edges,
vertices and faces, faces only as in the channels experiment of Section 5.2,
edges and faces, and vertices only) on the GPU against the oracle built with the same
selection: apply, PCG iterations and solution, for the FP64 and mixed paths.

Without vertices a floating subdomain's local Neumann matrix is singular; the
library factors A + sum rho_k c_k^T c_k over the averages lying in one z-plane
(an augmented Lagrangian, exact for the constrained problems), so the 12^3
mesh with 3^3 subdomains, whose centre box is floating, is in the cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bddc as orc  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402

_cache = {}


def _case(name, sel):
    if (name, sel) not in _cache:
        if name == "ragged":
            a = inputs.alpha_loguniform(14, 11, 9, -1, 1, 1)
            p = inputs.box_problem(14, 11, 9, [[5, 9], [4], [3, 6]], 3, alpha=a, selection=sel)
        else:   # 3^3 subdomains of 4^3: the centre one is floating
            a = inputs.alpha_loguniform(12, 12, 12, -1, 1, 2)
            p = inputs.box_problem(12, 12, 12, [[4, 8]] * 3, 2, alpha=a, selection=sel)
        _cache[(name, sel)] = (p, orc.build(p))
    return _cache[(name, sel)]


@pytest.mark.parametrize("name", ["ragged", "floating"])
@pytest.mark.parametrize("sel", ["ve", "vf", "v", "f", "ef"])
@pytest.mark.parametrize("precision,tol,dit", [("fp64", 1e-10, 1), ("mixed", 1e-8, 2)])
def test_selection_matches_oracle(name, sel, precision, tol, dit):
    from paper_2001_07289_gb300.bddc import BDDC
    p, ref = _case(name, sel)
    pre = BDDC.from_problem(p, precision=precision)
    info = pre.info()
    assert info["n_coarse"] == len(ref.sel)
    assert info["pinned_subdomains"] == (1 if (name == "floating" and "v" not in sel) else 0)
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_faces_only_coarse_basis_identity(precision, tol):
    """C_i Phi_i = I for the pinned (floating) subdomain with faces only, the
    basis being the exact saddle-point one with the augmented factor
    (checked against the oracle's)."""
    from paper_2001_07289_gb300.bddc import BDDC
    p, ref = _case("floating", "f")
    pre = BDDC.from_problem(p, precision=precision)
    centre = 13   # (1, 1, 1) of the 3^3 boxes
    phi, gid, node = pre.coarse_basis(centre)
    Phi_o, _, _ = ref.coarse_basis(centre)
    s = ref.subs[centre]
    pos = {int(v): k for k, v in enumerate(node)}
    loc = {int(v): k for k, v in enumerate(s.nodes)}
    Cs = np.zeros((len(s.obj), len(node)))
    for r, o in enumerate(s.obj):
        for v in ref.objs.nodes[o]:
            Cs[r, pos[int(v)]] = 1.0 / len(ref.objs.nodes[o])
    M = Cs @ phi
    perm = np.argmax(np.abs(M), axis=0)
    assert np.abs(M[perm, np.arange(len(perm))] - 1).max() < tol
    assert sorted(perm) == list(range(len(perm)))
    for b, v in enumerate(node):
        assert np.abs(phi[b] - Phi_o[loc[int(v)], perm]).max() <= tol * max(1.0, np.abs(Phi_o).max())
    pre.close()


def test_fewer_constraints_more_iterations():
    """Dropping constraints enlarges W-tilde: ve, vf and f need at least as
    many PCG iterations as vef, and vertices alone the most."""
    from paper_2001_07289_gb300.bddc import BDDC
    it = {}
    for sel in ("vef", "ve", "vf", "f", "v"):
        p = inputs.box_problem(24, 24, 24, [[8, 16]] * 3, 4, selection=sel)
        pre = BDDC.from_problem(p)
        _, st = pre.solve(torch.from_numpy(inputs.random_node_vector(24, 24, 24, 9)).cuda(), 1e-8)
        it[sel] = st["iterations"]
        pre.close()
    assert it["vef"] <= min(it["ve"], it["vf"], it["f"]), it
    assert it["v"] >= max(it["ve"], it["vf"]), it


def test_floating_without_plane_average_refused():
    """L = 1: every interface node is a vertex object, so faces only select
    nothing and the floating centre box has no row to pin with."""
    import paper_2001_07289_gb300.bddc as gb
    p = inputs.box_problem(12, 12, 12, [[4, 8]] * 3, 1, selection="f")
    with pytest.raises(gb.BddcError) as e:
        gb.BDDC.from_problem(p)
    assert e.value.code == gb.BDDC_ERR_UNSUPPORTED and "z-plane" in str(e.value)
