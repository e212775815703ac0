"""Size buckets of the apply's local solves and their tuned schedules.

A 20^3 mesh cut at element 14 on every axis has subdomains 14 and 6 elements
wide: the widest ones need a whole SM for their work vectors (bucket 0: the
14^3 box on the FP32 path, also the three 14 x 14 x 6 boxes with FP64
vectors), the others leave room for two CTAs per SM with the shallow
bulk-copy ring (bucket 1).  Every schedule of every bucket gives the same preconditioner:
the ring depth does not touch the arithmetic (bitwise equal), two or four
CTAs per subdomain only change the order in which partial sums meet (1e-12
FP64, 1e-6 mixed); and the tuned one matches the oracle (1e-10 FP64, 2e-5 mixed).
"""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bddc as orc  # noqa: E402
from paper_2001_07289_gb300 import inputs  # noqa: E402

if torch.cuda.is_available():
    import paper_2001_07289_gb300.bddc as gb  # noqa: E402


def problem(precision):
    a = inputs.alpha_loguniform(20, 20, 20, -1, 1, 12)
    return inputs.box_problem(20, 20, 20, [[14]] * 3, 4, alpha=a, precision=precision)


@pytest.mark.parametrize("precision,tol,otol,counts", [("fp64", 1e-12, 1e-10, [4, 4]), ("mixed", 1e-6, 2e-5, [1, 7])])
def test_buckets_schedules_agree(precision, tol, otol, counts):
    p = problem(precision)
    pre = gb.BDDC.from_problem(p)
    info = pre.info()
    assert info["n_buckets"] == 2
    assert info["bucket_subdomains"] == counts
    assert all(r in (4, 6) for r in info["bucket_ring"]) and all(c in (1, 2, 4) for c in info["bucket_ctas"])
    r = torch.from_numpy(inputs.random_node_vector(20, 20, 20, 3)).cuda()
    tuned = pre.apply(r).cpu().numpy()
    ref = orc.build(inputs.box_problem(20, 20, 20, p.cuts, p.L, alpha=p.alpha)).apply(r.cpu().numpy())
    assert np.abs(tuned - ref).max() <= otol * np.abs(ref).max()
    rings = {0: [6], 1: [6, 4]}
    with pytest.raises(gb.BddcError):
        pre.set_bucket_schedule(0, 4, 1)   # the wide box's vectors do not fit the shallow ring
    base = {}
    for r0, c0, r1, c1 in itertools.product(rings[0], (1, 2, 4), rings[1], (1, 2, 4)):
        pre.set_bucket_schedule(0, r0, c0)
        pre.set_bucket_schedule(1, r1, c1)
        z = pre.apply(r).cpu().numpy()
        key = (c0, c1)
        if key in base:
            assert np.array_equal(z, base[key]), (r0, c0, r1, c1)   # ring depth: same arithmetic
        else:
            base[key] = z
        assert np.abs(z - tuned).max() <= tol * np.abs(tuned).max()
    pre.close()


def test_bucketed_solve_matches_oracle():
    """PCG through both buckets (mixed path, graph) against the oracle."""
    p = problem("mixed")
    pre = gb.BDDC.from_problem(p, use_graph=True)
    x, st = pre.solve(torch.from_numpy(p.b).cuda(), 1e-10)
    ref = orc.build(inputs.box_problem(20, 20, 20, p.cuts, p.L, alpha=p.alpha))
    res = orc.pcg(ref.operator, ref.apply, p.b, 1e-10)
    assert st["converged"] and abs(st["iterations"] - res.iterations) <= 2
    assert np.linalg.norm(x.cpu().numpy() - res.x) / np.linalg.norm(res.x) <= 1e-8
    pre.close()
