"""Failure paths of the library, injected on the host (no GPU fault, trap or
hang is ever caused).

- A negated pivot: the test hook makes the next setups negate the first
  diagonal entry of one subdomain's assembled local matrix, so its
  factorisation meets a non-positive pivot; bddc_setup must return
  BDDC_ERR_NOT_SPD and name the subdomain.
- A bounded wait that runs out: the test hook lowers the number of tries after
  which the device waits (bulk copies of the streamed sweeps, tensor-core MMA
  completions) report a timeout to zero, so every wait reports; each wait
  still waits, bounded, for the work it covers, so the call returns
  BDDC_ERR_TIMEOUT with valid results and the handle stays usable.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2001_07289_gb300 import inputs  # noqa: E402

if torch.cuda.is_available():
    import paper_2001_07289_gb300.bddc as gb  # noqa: E402


def ragged(precision):
    a = inputs.alpha_loguniform(14, 11, 9, -1, 1, 1)
    return inputs.box_problem(14, 11, 9, [[5, 9], [4], [3, 6]], 3, alpha=a, precision=precision)


@pytest.fixture
def hooks():
    yield gb
    gb.debug_inject(gb.BDDC_DEBUG_CLEAR)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("problem", ["neumann", "dirichlet"])
def test_negated_pivot_reports_not_spd(hooks, precision, problem):
    p = ragged(precision)
    what = gb.BDDC_DEBUG_NEGATE_NEUMANN_PIVOT if problem == "neumann" else gb.BDDC_DEBUG_NEGATE_DIRICHLET_PIVOT
    sub = 7    # (sx, sy, sz) = (1, 0, 1): widths 4 x 4 x 3, interior nodes present
    gb.debug_inject(what, sub)
    with pytest.raises(gb.BddcError) as e:
        gb.BDDC.from_problem(p)
    assert e.value.code == gb.BDDC_ERR_NOT_SPD
    assert f"{problem.capitalize()} factor of subdomain {sub}" in str(e.value)
    gb.debug_inject(gb.BDDC_DEBUG_CLEAR)
    # later setups are unaffected
    pre = gb.BDDC.from_problem(p)
    _, st = pre.solve(torch.from_numpy(p.b).cuda(), 1e-10)
    assert st["converged"]
    pre.close()


def test_debug_hook_rejects_unknown_requests():
    with pytest.raises(gb.BddcError) as e:
        gb.debug_inject(99, 0)
    assert e.value.code == gb.BDDC_ERR_ARG


def _pcg(pre, b, x):
    st = gb.Stats(0, 0, 0.0, 0.0, None, None, 0, 0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = gb.lib.pcg_solve(pre._handle, gb._ptr(b), gb._ptr(x), 1e-10, ctypes.byref(st), stream)
    torch.cuda.synchronize()
    return code, st.iterations


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bounded_wait_timeout_is_reported(hooks, precision):
    p = ragged(precision)
    pre = gb.BDDC.from_problem(p)
    b = torch.from_numpy(inputs.random_node_vector(14, 11, 9, 8)).cuda()
    x_ref = torch.empty_like(b)
    code, it_ref = _pcg(pre, b, x_ref)
    assert code == gb.BDDC_OK
    gb.debug_inject(gb.BDDC_DEBUG_WAIT_TRIES, 0)
    x = torch.full_like(b, np.nan)
    code, it = _pcg(pre, b, x)
    assert code == gb.BDDC_ERR_TIMEOUT
    assert "bounded device wait" in gb.lib.bddc_last_error(pre._handle).decode()
    # every wait still covered its copy: the solve itself is unchanged
    assert it == it_ref
    assert torch.equal(x, x_ref)
    if precision == "mixed":
        # a setup also reports it: the tensor-core solves of the FP32 path
        # wait on bulk copies and MMA completions
        with pytest.raises(gb.BddcError) as e:
            gb.BDDC.from_problem(p)
        assert e.value.code == gb.BDDC_ERR_TIMEOUT
    gb.debug_inject(gb.BDDC_DEBUG_CLEAR)
    # the status was cleared when it was read: the handle works again
    x2 = torch.empty_like(b)
    code, it2 = _pcg(pre, b, x2)
    assert code == gb.BDDC_OK and it2 == it_ref
    assert torch.equal(x2, x_ref)
    pre.close()
