"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (written per test): the FP64 path computes the same quantities as
the oracle with a different but backward-stable elimination order (plane-block
Cholesky with explicit inverse diagonal blocks against sparse LU), so
elementwise agreement is at the level of the condition numbers of the local
problems times 1e-16; 1e-10 relative to the vector's max is used for B r and
the coarse basis.  The mixed path runs the local factors and solves in FP32
(unit roundoff 6e-8), so its preconditioner agrees to ~1e-5; its PCG solution
is checked against the FP64 oracle at <= 1e-8 (the outer PCG is FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bddc as orc  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402

if torch.cuda.is_available():
    from paper_2001_07289_gb300.bddc import BDDC, BddcError, solve_host  # noqa: E402
    import paper_2001_07289_gb300.bddc as gb  # noqa: E402


def ragged(L=3, weights="card", seed=1, precision="fp64"):
    """14 x 11 x 9 elements, uneven boxes (widths 5,4,5 / 4,7 / 3,3,3)."""
    a = inputs.alpha_loguniform(14, 11, 9, -1, 1, seed)
    return inputs.box_problem(14, 11, 9, [[5, 9], [4], [3, 6]], L, alpha=a, weights=weights,
                              precision=precision)


CASES = {
    "poisson16": lambda prec: inputs.workload(0, precision=prec),
    "poisson16_L2": lambda prec: inputs.workload(0, L=2, precision=prec),
    "ragged_L3": lambda prec: ragged(precision=prec),
    "ragged_rho_L2": lambda prec: ragged(L=2, weights="rho", seed=3, precision=prec),
    "blocks24_rho": lambda prec: inputs.box_problem(
        24, 24, 24, [[12]] * 3, 4, alpha=inputs.alpha_blocks(24, 24, 24, 4, 1e6, 0.3, 7), weights="rho",
        precision=prec),
    "jitter_L1": lambda prec: inputs.box_problem(
        10, 9, 8, [[3, 7], [2, 5], [4]], 1, alpha=inputs.alpha_loguniform(10, 9, 8, -2, 2, 4), precision=prec),
    "one_axis": lambda prec: inputs.box_problem(12, 6, 6, [[4, 8], [], []], 4, precision=prec),
    "single_subdomain": lambda prec: inputs.box_problem(8, 8, 8, [[], [], []], 4, precision=prec),
    "width_one": lambda prec: inputs.box_problem(8, 8, 8, [[1, 2, 6], [4], [7]], 2, precision=prec),
}

_oracle_cache = {}


def oracle_for(name):
    if name not in _oracle_cache:
        p = CASES[name]("fp64")
        _oracle_cache[name] = (p, orc.build(p))
    return _oracle_cache[name]


def gpu(p, precision):
    return BDDC.from_problem(p, precision=precision)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# --------------------------------------------------------------------------
def test_library_exports():
    for name in gb.EXPORTS:
        assert hasattr(gb.lib, name)


@pytest.mark.parametrize("name", ["poisson16", "ragged_L3", "jitter_L1"])
def test_operator_matches_oracle(name):
    p, ref = oracle_for(name)
    pre = gpu(p, "fp64")
    x = inputs.random_node_vector(p.nx, p.ny, p.nz, 17)
    x_bnd = x + 5.0 * ref.bnd          # Dirichlet entries must be ignored
    y = pre.operator(cu(x_bnd)).cpu().numpy()
    want = ref.operator(x)
    assert np.abs(y - want).max() <= 1e-13 * np.abs(want).max()
    assert np.all(y[ref.bnd] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_space_size(name):
    p, ref = oracle_for(name)
    pre = gpu(p, "fp64")
    info = pre.info()
    assert info["n_coarse"] == ref.n_coarse
    assert info["n_sub"] == len(ref.subs)


def _perm_from_constraints(ref, i, phi, node):
    """Columns of the GPU basis matched to the oracle's objects through
    C_i Phi_i = I (C_i restricted to the box surface holds every object)."""
    s = ref.subs[i]
    pos = {int(v): k for k, v in enumerate(node)}
    Cs = np.zeros((len(s.obj), len(node)))
    for r, o in enumerate(s.obj):
        on = ref.objs.nodes[o]
        for v in on:
            Cs[r, pos[int(v)]] = 1.0 / len(on)
    M = Cs @ phi
    perm = np.argmax(np.abs(M), axis=0)
    return M, perm


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
@pytest.mark.parametrize("name", ["poisson16", "ragged_L3", "ragged_rho_L2", "jitter_L1"])
def test_coarse_basis_matches_oracle(name, precision, tol):
    p, ref = oracle_for(name)
    pre = gpu(p, precision)
    for i, s in enumerate(ref.subs):
        phi, gid, node = pre.coarse_basis(i)
        M, perm = _perm_from_constraints(ref, i, phi, node)
        assert np.abs(M[perm, np.arange(len(perm))] - 1).max() < tol      # C_i Phi_i = I
        assert sorted(perm) == list(range(len(perm)))
        Phi_o, _, _ = ref.coarse_basis(i)
        loc = {int(v): k for k, v in enumerate(s.nodes)}
        for b, v in enumerate(node):
            if int(v) in loc:
                row = Phi_o[loc[int(v)], perm]
                assert np.abs(phi[b] - row).max() <= tol * max(1.0, np.abs(Phi_o).max()), (i, b)
            else:
                assert np.all(phi[b] == 0)   # Dirichlet-boundary node


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
@pytest.mark.parametrize("name", list(CASES))
def test_apply_matches_oracle(name, precision, tol):
    p, ref = oracle_for(name)
    pre = gpu(p, precision)
    for seed in (3, 4):
        r = inputs.random_node_vector(p.nx, p.ny, p.nz, seed) + 3.0 * ref.bnd
        z = pre.apply(cu(r)).cpu().numpy()
        want = ref.apply(r)
        assert np.abs(z - want).max() <= tol * np.abs(want).max(), (name, np.abs(z - want).max())
        assert np.all(z[ref.bnd] == 0.0)


@pytest.mark.parametrize("precision,tol,dit", [("fp64", 1e-10, 1), ("mixed", 1e-8, 2)])
@pytest.mark.parametrize("name", ["poisson16", "ragged_L3", "ragged_rho_L2", "blocks24_rho", "jitter_L1",
                                  "single_subdomain", "width_one"])
def test_pcg_matches_oracle(name, precision, tol, dit):
    p, ref = oracle_for(name)
    pre = gpu(p, precision)
    b = p.b
    # f = 1 on the symmetric 16^3 mesh lies where B A = I exactly, so the FP64
    # oracle stops after one step; FP32 rounding in the mixed B (~1e-7) needs a
    # few more to reach 1e-10 whatever the implementation, so a random load is
    # used there (and on the ragged mesh).
    if name == "ragged_L3" or (name == "poisson16" and precision == "mixed"):
        b = inputs.random_node_vector(p.nx, p.ny, p.nz, 8)
    x, st = pre.solve(cu(b), 1e-10)
    res = orc.pcg(ref.operator, ref.apply, b, 1e-10)
    xg = x.cpu().numpy()
    assert st["converged"] and res.converged
    assert abs(st["iterations"] - res.iterations) <= dit, (st["iterations"], res.iterations)
    err = np.linalg.norm(xg - res.x) / np.linalg.norm(res.x)
    assert err <= tol, err
    # the GPU's own residual claim holds in the oracle's arithmetic
    assert np.linalg.norm(b * (1 - ref.bnd) - ref.operator(xg)) <= 1.01e-10 * np.linalg.norm(b * (1 - ref.bnd))


def test_pcg_coefficients_and_lanczos():
    p, ref = oracle_for("ragged_L3")
    pre = gpu(p, "fp64")
    b = inputs.random_node_vector(p.nx, p.ny, p.nz, 8)
    _, st = pre.solve(cu(b), 1e-12)
    res = orc.pcg(ref.operator, ref.apply, b, 1e-12)
    n = min(len(st["alphas"]), len(res.alphas))
    assert np.abs(st["alphas"][:n] - res.alphas[:n]).max() <= 1e-8 * np.abs(res.alphas).max()
    lo, hi = orc.lanczos_extremes(st["alphas"], st["betas"])
    assert lo >= 1 - 1e-10


def test_all_gamma_primal_is_exact_inverse():
    """L = 2h, tensor sub-partition: B = A^{-1}, PCG takes one iteration."""
    p, ref = oracle_for("poisson16_L2")
    pre = gpu(p, "fp64")
    x = inputs.random_node_vector(16, 16, 16, 9)
    z = pre.apply(pre.operator(cu(x))).cpu().numpy()
    assert np.abs(z - x).max() <= 1e-11 * np.abs(x).max()
    _, st = pre.solve(cu(p.b), 1e-10)
    assert st["iterations"] == 1


def test_deterministic_repeat():
    p, _ = oracle_for("ragged_rho_L2")
    out = []
    for _ in range(2):
        pre = gpu(p, "mixed")
        x, _ = pre.solve(cu(p.b), 1e-10)
        out.append(x.cpu().numpy())
        pre.close()
    assert np.array_equal(out[0], out[1])


def test_gradient_matches_oracle_and_euler_identity():
    p = inputs.box_problem(12, 10, 8, [[6], [5], [4]], 2, alpha=np.exp(inputs.gaussian_field(12, 10, 8, 0.2, 5)))
    pre = gpu(p, "fp64")
    rng_u = inputs.random_node_vector(12, 10, 8, 1)
    rng_l = inputs.random_node_vector(12, 10, 8, 2)
    g = pre.gradient(cu(rng_u), cu(rng_l)).cpu().numpy()
    want = orc.gradient(12, 10, 8, p.h, rng_u, rng_l)
    assert np.abs(g - want).max() <= 1e-13 * np.abs(want).max()
    # Euler identity on a solved pair
    b = cu(p.b)
    u, _ = pre.solve(b, 1e-13)
    lam, _ = pre.solve(u, 1e-13)
    gg = pre.gradient(u, lam).cpu().numpy()
    lhs = np.sum(p.alpha * gg)
    rhs = -float(lam.cpu().numpy() @ p.b)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_solve_host_matches_device_path():
    p, ref = oracle_for("ragged_L3")
    x_host, st = solve_host(p.nx, p.ny, p.nz, p.cuts, p.L, p.alpha, p.b, 1e-10)
    pre = gpu(p, "fp64")
    x_dev, st2 = pre.solve(cu(p.b), 1e-10)
    assert st["iterations"] == st2["iterations"]
    assert np.array_equal(x_host, x_dev.cpu().numpy())


def test_errors_are_reported():
    p = inputs.workload(0)
    bad = p.alpha.copy()
    bad[17] = -1.0
    with pytest.raises(BddcError) as e:
        BDDC(16, 16, 16, p.cuts, 4, cu(bad))
    assert e.value.code == gb.BDDC_ERR_ARG
    bad[17] = np.nan
    with pytest.raises(BddcError):
        BDDC(16, 16, 16, p.cuts, 4, cu(bad))
    with pytest.raises(BddcError) as e:
        BDDC(16, 16, 16, [[8, 8], [8], [8]], 4, cu(p.alpha))
    assert e.value.code == gb.BDDC_ERR_ARG
    with pytest.raises(BddcError):
        BDDC(16, 16, 16, p.cuts, 0, cu(p.alpha))
    pre = BDDC(16, 16, 16, p.cuts, 4, cu(p.alpha), maxit=1)
    b = cu(inputs.random_node_vector(16, 16, 16, 2))
    with pytest.raises(BddcError) as e:
        pre.solve(b, 1e-12)
    assert e.value.code == gb.BDDC_ERR_NOCONV
    x, st = pre.solve(b, 1e-12, raise_on_noconv=False)
    assert st["iterations"] == 1 and not st["converged"]


def test_zero_rhs():
    p = inputs.workload(0)
    pre = gpu(p, "fp64")
    x, st = pre.solve(torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda"), 1e-10)
    assert st["iterations"] == 0 and st["converged"]
    assert torch.all(x == 0)


@pytest.mark.parametrize("name", ["poisson16", "ragged_L3", "jitter_L1"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_apply_schedules_agree(name, precision, tol):
    """The apply's local solves on one CTA per subdomain and on clusters of
    two or four CTAs (rows of every slot split, partial sums exchanged through
    distributed shared memory) give the same preconditioner up to summation
    order, on the same handle; the autotuned choice is one of them (jitter_L1
    has planes of a few nodes, where four CTAs leave some with no rows)."""
    p, _ = oracle_for(name)
    pre = gpu(p, precision)
    assert pre.info()["apply_cluster"] in (1, 2, 4)
    r = cu(inputs.random_node_vector(p.nx, p.ny, p.nz, 21))
    out = {}
    for c in (1, 2, 4):
        pre.set_apply_schedule(c)
        out[c] = pre.apply(r).cpu().numpy()
        x, st = pre.solve(cu(p.b), 1e-10, raise_on_noconv=False)
        out[(c, "it")] = st["iterations"]
    for c in (2, 4):
        assert np.abs(out[1] - out[c]).max() <= tol * np.abs(out[1]).max()
        assert abs(out[(1, "it")] - out[(c, "it")]) <= 1
    with pytest.raises(BddcError):
        pre.set_apply_schedule(3)
