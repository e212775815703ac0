"""The paper's experiments and the full-size workloads on the GPU.

Table 1 (Section 5.1) iteration counts at true size; the heterogeneous
(channels96), jittered (jitter128) and adjoint (adjoint64) workloads at full
size, checked through
properties that hold at any size in the oracle's arithmetic (residual of the
returned solution, agreement of the mixed and FP64 paths, the gradient's Euler
identity and central differences); the adjoint through the autograd Function
against the oracle's gradient on a small mesh.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bddc as orc, fem  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402
from tests.golden import read as golden  # noqa: E402

if torch.cuda.is_available():
    from paper_2001_07289_gb300.bddc import BDDC, BddcSolve  # noqa: E402


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("k", [4, 8])
def test_table1_iterations(k):
    """(10k)^3 hexahedra, 10^3 subdomains of k^3, f = 1, residual reduced by
    1e6: BDDC-SO(vef) with L/h = 4 and BDDC(vef) (L = k); counts within one of
    Table 1 (the paper leaves averaging details open, so +-1)."""
    it = golden.table1_iterations()
    sizes = golden.table1_coarse_sizes()
    n = 10 * k
    cuts = [inputs.uniform_cuts(n, 10)] * 3
    b = cu(inputs.rhs_constant(n, n, n, 1.0 / n))
    for method, L in (("BDDC-SO(vef)", 4), ("BDDC(vef)", k)):
        pre = BDDC(n, n, n, cuts, L, cu(np.ones(n ** 3)), precision="fp64")
        assert pre.info()["n_coarse"] == sizes[(method, k)]
        _, st = pre.solve(b, 1e-6)
        assert abs(st["iterations"] - it[(method, k)]) <= 1, (method, k, st["iterations"])
        pre.close()


def test_channels96_full_size():
    """Workload 2 (96^3, 8^3 subdomains, alpha in {1, 1e6} per 4^3 block,
    rho-weights, mixed, rtol 1e-8): the mixed solution's residual in the
    oracle's arithmetic, few iterations despite the 1e6 contrast, and agreement
    with the FP64 path."""
    p = inputs.workload(2)
    a, b = cu(p.alpha), cu(p.b)
    pre = BDDC.from_problem(p, alpha=a, precision="mixed")
    x, st = pre.solve(b, p.rtol)
    assert st["converged"] and st["iterations"] <= 20
    xg = x.cpu().numpy()
    A = fem.assemble(p.nx, p.ny, p.nz, p.h, p.alpha).tocsr()
    bnd = fem.boundary_node_mask(p.nx, p.ny, p.nz)
    res = np.where(bnd, 0.0, p.b - A @ np.where(bnd, 0.0, xg))
    assert np.linalg.norm(res) <= 1.01 * p.rtol * np.linalg.norm(p.b)
    pre.close()
    # at rtol 1e-8 and a 1e6 contrast two valid answers may differ by more
    # than 1e-8, so the paths are compared solved to 1e-12
    pre64 = BDDC.from_problem(p, alpha=a, precision="fp64")
    x64, st64 = pre64.solve(b, 1e-12)
    x32, st32 = BDDC.from_problem(p, alpha=a, precision="mixed").solve(b, 1e-12)
    assert abs(st32["iterations"] - st64["iterations"]) <= 3, (st32["iterations"], st64["iterations"])
    x64 = x64.cpu().numpy()
    err = np.linalg.norm(x32.cpu().numpy() - x64) / np.linalg.norm(x64)
    assert err <= 1e-8, err


def test_adjoint_autograd_matches_oracle_small():
    """BddcSolve backward against the oracle's adjoint gradient (direct solves)
    on a 12^3 mesh with a Gaussian-field coefficient; relative error <= 1e-6."""
    n = 12
    p = inputs.box_problem(n, n, n, [[6]] * 3, 3, alpha=np.exp(inputs.gaussian_field(n, n, n, 0.2, 11)))
    uobs = inputs.random_node_vector(n, n, n, 12) * 1e-3
    bnd = fem.boundary_node_mask(n, n, n)
    alpha = cu(p.alpha).requires_grad_(True)
    u = BddcSolve.apply(alpha, cu(p.b), p, 1e-13)
    J = 0.5 * torch.sum(torch.where(cu(bnd), 0.0, u - cu(uobs)) ** 2)
    J.backward()
    g = alpha.grad.cpu().numpy()
    uo = orc.direct_solve(n, n, n, p.h, p.alpha, p.b)
    lam = orc.direct_solve(n, n, n, p.h, p.alpha, np.where(bnd, 0.0, uo - uobs))
    want = orc.gradient(n, n, n, p.h, uo, lam)
    assert np.abs(g - want).max() <= 1e-6 * np.abs(want).max()


def test_adjoint_autograd_matches_oracle_32():
    """The same at 32^3 with 4^3 subdomains of 8^3 and L = 4h: the gradient
    through the autograd Function (forward and adjoint PCG to 1e-13 on the
    same handle) against the oracle's adjoint gradient from sparse direct
    solves; relative error <= 1e-6."""
    n = 32
    p = inputs.box_problem(n, n, n, [inputs.uniform_cuts(n, 4)] * 3, 4,
                           alpha=np.exp(inputs.gaussian_field(n, n, n, 0.1, 21)))
    uobs = inputs.random_node_vector(n, n, n, 22) * 1e-3
    bnd = fem.boundary_node_mask(n, n, n)
    alpha = cu(p.alpha).requires_grad_(True)
    u = BddcSolve.apply(alpha, cu(p.b), p, 1e-13)
    J = 0.5 * torch.sum(torch.where(cu(bnd), 0.0, u - cu(uobs)) ** 2)
    J.backward()
    g = alpha.grad.cpu().numpy()
    uo = orc.direct_solve(n, n, n, p.h, p.alpha, p.b)
    lam = orc.direct_solve(n, n, n, p.h, p.alpha, np.where(bnd, 0.0, uo - uobs))
    want = orc.gradient(n, n, n, p.h, uo, lam)
    assert np.abs(g - want).max() <= 1e-6 * np.abs(want).max()


def test_adjoint64_full_size():
    """Workload 4 (64^3, 4^3 subdomains, log alpha a Gaussian field, FP64):
    u_obs from a second field plus 1 % noise; the gradient from the autograd
    Function satisfies sum_e alpha_e g_e = -lambda^T b and matches central
    differences in theta = log alpha (step 1e-6) along all 20 seeded
    directions of the workload."""
    p = inputs.workload(4)
    n = p.nx
    bnd = fem.boundary_node_mask(n, n, n)
    b = cu(p.b)
    # observation: forward solution for the second field, 1 % noise
    pobs = BDDC(n, n, n, p.cuts, p.L, cu(inputs.observation_field_alpha(n)), precision="fp64")
    u2, _ = pobs.solve(b, 1e-13)
    pobs.close()
    uobs = u2.cpu().numpy() * (1.0 + 0.01 * inputs.observation_noise(p.n_nodes))
    alpha = cu(p.alpha).requires_grad_(True)
    u = BddcSolve.apply(alpha, b, p, 1e-13)
    J = 0.5 * torch.sum(torch.where(cu(bnd), 0.0, u - cu(uobs)) ** 2)
    J.backward()
    g = alpha.grad.cpu().numpy()
    # Euler identity with the adjoint state recomputed on the same handle
    pre = BDDC.from_problem(p, alpha=cu(p.alpha), precision="fp64")
    lam, _ = pre.solve(cu(np.where(bnd, 0.0, u.detach().cpu().numpy() - uobs)), 1e-13)
    lhs = float(np.sum(p.alpha * g))
    rhs = -float(lam.cpu().numpy() @ p.b)
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs)
    pre.close()
    dirs = inputs.fd_directions(p.n_elems, count=20)
    assert dirs.shape == (20, p.n_elems)
    t = 1e-6
    for d in dirs:
        us = []
        for sgn in (1.0, -1.0):
            pp = BDDC.from_problem(p, alpha=cu(p.alpha * np.exp(sgn * t * d)), precision="fp64")
            u_s, _ = pp.solve(b, 1e-14, raise_on_noconv=False)
            us.append(np.where(bnd, 0.0, u_s.cpu().numpy()))
            pp.close()
        # (J(+t) - J(-t)) / 2t in the product form 1/2 sum (u+ - u-)(u+ + u- - 2 u_obs):
        # the same number without subtracting two values of J (about 10 each)
        # that agree to nine digits
        ob = np.where(bnd, 0.0, uobs)
        fd = 0.5 * float((us[0] - us[1]) @ (us[0] + us[1] - 2.0 * ob)) / (2 * t)
        an = float(np.sum(g * p.alpha * d))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def _jitter(n, parts, seed, precision):
    """The jitter128 recipe (jittered cuts, alpha = 10^U[-2,2] per element,
    f = 1, L = 4) on an n^3 mesh with parts^3 subdomains."""
    cuts = [inputs.jittered_cuts(n, parts, seed + d) for d in range(3)]
    a = inputs.alpha_loguniform(n, n, n, -2.0, 2.0, seed + 3)
    return inputs.box_problem(n, n, n, cuts, 4, alpha=a, rtol=1e-10, precision=precision)


def test_jitter_recipe_fp64_matches_oracle():
    """The jitter128 input recipe at 24^3 (3^3 jittered subdomains), run with
    the PCG loop as a CUDA graph, against the oracle's PCG at rtol 1e-10
    (about a hundred iterations: alpha is not constant on subobjects): the
    FP64 path follows the oracle's iterates, relative error <= 1e-10 and
    iteration counts within 1."""
    p = _jitter(24, 3, 91, "fp64")
    ref = orc.build(p)
    res = orc.pcg(ref.operator, ref.apply, p.b, p.rtol)
    pre = BDDC.from_problem(p, alpha=cu(p.alpha), use_graph=True)
    x, st = pre.solve(cu(p.b), p.rtol)
    pre.close()
    assert st["converged"] and res.converged
    assert abs(st["iterations"] - res.iterations) <= 1, (st["iterations"], res.iterations)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - res.x) / np.linalg.norm(res.x) <= 1e-10
    bf = p.b * (1 - ref.bnd)
    assert np.linalg.norm(bf - ref.operator(xg)) <= 1.01 * p.rtol * np.linalg.norm(bf)


@pytest.mark.parametrize("beta", ["standard", "flexible"])
def test_jitter_recipe_mixed_matches_oracle(beta):
    """The same recipe on the mixed path (FP32 local factors and solves),
    compared as the tolerance reading for configurations that cannot meet
    1e-8 at their own rtol prescribes: both solved to rtol 1e-12, relative
    error <= 1e-8, the GPU's residual claim checked in the oracle's
    arithmetic.  Iterations at the workload's rtol 1e-10: the FP32 local
    solves add a measured 11 to the oracle's 102 (113 standard, 114 flexible
    beta); storing only the Neumann factor, or only Phi, of the FP64 path in
    FP32 already adds 8 and 7 (the constrained Neumann correction
    Phi (u_c - C y) + y cancels large near-kernel components of y when alpha
    varies by 1e4 between elements), so the window is 12 + 1."""
    p = _jitter(24, 3, 91, "mixed")
    ref = orc.build(inputs.box_problem(p.nx, p.ny, p.nz, p.cuts, p.L, alpha=p.alpha))
    pre = BDDC.from_problem(p, alpha=cu(p.alpha), use_graph=True, beta=beta)
    res10 = orc.pcg(ref.operator, ref.apply, p.b, 1e-10)
    _, st = pre.solve(cu(p.b), 1e-10)
    assert st["converged"] and res10.converged
    assert 0 <= st["iterations"] - res10.iterations <= 13, (st["iterations"], res10.iterations)
    res = orc.pcg(ref.operator, ref.apply, p.b, 1e-12)
    x, st = pre.solve(cu(p.b), 1e-12)
    pre.close()
    assert st["converged"] and res.converged
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - res.x) / np.linalg.norm(res.x) <= 1e-8
    bf = p.b * (1 - ref.bnd)
    assert np.linalg.norm(bf - ref.operator(xg)) <= 1.01e-12 * np.linalg.norm(bf)


def test_jitter128_full_size():
    """Workload jitter128 (128^3, 16^3 jittered subdomains of widths 5..11,
    alpha = 10^U[-2,2] per element, L = 4h, mixed, PCG as a CUDA graph, rtol
    1e-10): the coarse size equals the host analysis (itself checked against
    Table 1 and the oracle's object counts), and the returned solution meets
    the tolerance in the oracle's arithmetic (element-by-element operator).
    alpha varies per element, outside Theorem 1's assumption of a coefficient
    constant on each subobject, so PCG needs a few hundred iterations (253 with
    the mixed path, 239 with FP64 on a GB300); the bound only guards against a
    regression."""
    from paper_2001_07289_gb300.bddc import analyze
    p = inputs.workload(3)
    pre = BDDC.from_problem(p, alpha=cu(p.alpha), use_graph=True, maxit=400)
    assert pre.info()["n_coarse"] == analyze(p.nx, p.ny, p.nz, p.cuts, p.L)["n_coarse"]
    x, st = pre.solve(cu(p.b), p.rtol)
    pre.close()
    assert st["converged"] and st["iterations"] <= 300, st["iterations"]
    xg = x.cpu().numpy()
    r = p.b * (1 - fem.boundary_node_mask(p.nx, p.ny, p.nz)) - fem.apply_operator_by_elements(
        p.nx, p.ny, p.nz, p.h, p.alpha, xg)
    bn = np.linalg.norm(p.b * (1 - fem.boundary_node_mask(p.nx, p.ny, p.nz)))
    assert np.linalg.norm(r) <= 1.01 * p.rtol * bn


@pytest.mark.parametrize("L,n_coarse,maxit", [(4, None, 400), (2, 643455, 400)])
def test_jitter128_multilevel_full_size(L, n_coarse, maxit):
    """jitter128 with the multilevel coarse level (blocks of 2^3 subdomains,
    Section 6), mixed path, PCG as a CUDA graph, rtol 1e-10, at L = 4h and at
    L = 2h, where the coarse problem has 643,455 DOFs (every interface DOF
    primal; too large for the exact coarse factorisation): 512 blocks and
    2,863 level-2 DOFs, and the returned solution meets the tolerance in the
    oracle's arithmetic.  Measured on a GB300: 260 iterations at L = 4h, 290
    at L = 2h (the coarse level is then preconditioned, not exact)."""
    from paper_2001_07289_gb300.bddc import analyze
    p = inputs.workload(3, L=L)
    pre = BDDC.from_problem(p, alpha=cu(p.alpha), use_graph=True, maxit=maxit, ml_block=2)
    info = pre.info()
    assert info["n_coarse"] == analyze(p.nx, p.ny, p.nz, p.cuts, p.L)["n_coarse"]
    if n_coarse:
        assert info["n_coarse"] == n_coarse
    assert (info["ml_blocks"], info["ml_coarse2"]) == (512, 2863)
    x, st = pre.solve(cu(p.b), p.rtol)
    pre.close()
    assert st["converged"] and st["iterations"] <= 330, st["iterations"]
    xg = x.cpu().numpy()
    mask = 1 - fem.boundary_node_mask(p.nx, p.ny, p.nz)
    r = p.b * mask - fem.apply_operator_by_elements(p.nx, p.ny, p.nz, p.h, p.alpha, xg)
    assert np.linalg.norm(r) <= 1.01 * p.rtol * np.linalg.norm(p.b * mask)
