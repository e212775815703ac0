"""PCG with the loop captured as one CUDA graph (options.use_graph = 1).

The graph's while body launches the same kernels in the same order as the
host-driven loop, so both modes must return bitwise identical iterates,
iteration counts and CG coefficients; the device-side stopping test (Section
5's residual rule) must end the loop at the tolerance, at maxit, or at once
for b = 0.  Also checked against the oracle's iteration count."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2001_07289_gb300 import inputs  # noqa: E402


def _pair(p, **kw):
    import paper_2001_07289_gb300.bddc as gb
    a = torch.from_numpy(p.alpha).cuda()
    return (gb.BDDC.from_problem(p, alpha=a, use_graph=False, **kw),
            gb.BDDC.from_problem(p, alpha=a, use_graph=True, **kw))


CASES = {
    "poisson16_fp64": lambda: inputs.workload(0),
    "ragged_mixed": lambda: inputs.box_problem(
        17, 13, 11, [[5, 11], [6], [4, 8]], 3, alpha=inputs.alpha_loguniform(17, 13, 11, -2, 2, 7),
        precision="mixed"),
    "rho_fp64": lambda: inputs.box_problem(
        16, 16, 16, [[8]] * 3, 4, alpha=inputs.alpha_blocks(16, 16, 16, 4, 1e4, 0.3, 8), weights="rho"),
}


@pytest.mark.parametrize("beta", ["standard", "flexible"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_graph_equals_host_loop(name, beta):
    p = CASES[name]()
    host, graph = _pair(p, beta=beta)
    b = torch.from_numpy(p.b).cuda()
    xh, sh = host.solve(b, p.rtol)
    for rep in range(2):   # the second solve reuses the captured graph
        xg, sg = graph.solve(b, p.rtol)
        assert sg["iterations"] == sh["iterations"]
        assert sg["converged"] and sh["converged"]
        assert torch.equal(xg, xh)
        assert np.array_equal(sg["alphas"], sh["alphas"])
        assert np.array_equal(sg["betas"], sh["betas"])
        assert sg["r_norm"] == sh["r_norm"] and sg["r0_norm"] == sh["r0_norm"]
    host.close()
    graph.close()


def test_graph_iterations_match_oracle():
    from oracle import bddc as ob
    p = CASES["ragged_mixed"]()
    p_fp64 = inputs.box_problem(p.nx, p.ny, p.nz, p.cuts, p.L, alpha=p.alpha, precision="fp64")
    op = ob.build(p_fp64)
    ref = ob.pcg(op.operator, op.apply, p_fp64.b, p_fp64.rtol)
    host, graph = _pair(p_fp64)
    host.close()
    x, s = graph.solve(torch.from_numpy(p_fp64.b).cuda(), p_fp64.rtol)
    assert abs(s["iterations"] - ref.iterations) <= 1
    err = np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-9
    graph.close()


def test_graph_new_rtol_and_rhs_reuse_graph():
    """The tolerance and b are inputs of each solve, not of the capture."""
    p = CASES["rho_fp64"]()
    host, graph = _pair(p)
    for seed, rtol in ((1, 1e-6), (2, 1e-11), (3, 1e-3)):
        b = torch.from_numpy(inputs.random_node_vector(p.nx, p.ny, p.nz, seed)).cuda()
        xh, sh = host.solve(b, rtol)
        xg, sg = graph.solve(b, rtol)
        assert sg["iterations"] == sh["iterations"]
        assert torch.equal(xg, xh)
        assert sg["r_norm"] <= rtol * sg["r0_norm"]
    host.close()
    graph.close()


def test_graph_stops_at_maxit():
    import paper_2001_07289_gb300.bddc as gb
    p = CASES["ragged_mixed"]()
    host, graph = _pair(p, maxit=3)
    b = torch.from_numpy(p.b).cuda()
    xh, sh = host.solve(b, 1e-14, raise_on_noconv=False)
    xg, sg = graph.solve(b, 1e-14, raise_on_noconv=False)
    assert sh["status"] == sg["status"] == gb.BDDC_ERR_NOCONV
    assert sg["iterations"] == sh["iterations"] == 3
    assert torch.equal(xg, xh)
    host.close()
    graph.close()


def test_graph_zero_rhs():
    p = CASES["poisson16_fp64"]()
    host, graph = _pair(p)
    host.close()
    b = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    x = torch.full_like(b, 7.0)
    x, s = graph.solve(b, 1e-10, out=x)
    assert s["iterations"] == 0 and s["converged"]
    assert torch.count_nonzero(x).item() == 0
    graph.close()
