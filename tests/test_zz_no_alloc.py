"""bddc_apply_noalloc: the allocation-free preconditioner apply.

It serves callers that must not allocate device memory while they apply the
preconditioner; it takes its work vectors from the library's fixed device
array.  Checked through the C ABI against bddc_apply on the same handle, on two
calls in a row (the array keeps the previous call's contents, so the second
call shows that everything that must start at zero is cleared), for the FP64
and the mixed path.  The file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2001_07289_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-10)])
def test_apply_noalloc_matches_apply(precision, tol):
    import paper_2001_07289_gb300.bddc as gb
    a = inputs.alpha_loguniform(14, 11, 9, -1, 1, 1)
    p = inputs.box_problem(14, 11, 9, [[5, 9], [4], [3, 6]], 3, alpha=a, precision=precision)
    pre = gb.BDDC.from_problem(p)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    r1 = torch.from_numpy(inputs.random_node_vector(14, 11, 9, 3)).cuda()
    r2 = torch.from_numpy(inputs.random_node_vector(14, 11, 9, 4) + 2.0).cuda()
    # first call on this device looks up the array's address
    z = torch.empty_like(r1)
    assert gb.lib.bddc_apply_noalloc(pre._handle, gb._ptr(r1), gb._ptr(z), stream) == 0
    # every tensor of the test exists before the device's free memory is read,
    # and handles that earlier tests dropped are freed now, not during the loop
    outs = [(torch.empty_like(r1), torch.full_like(r1, np.nan)) for _ in range(2)]
    gc.collect()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for r, (want, got) in zip((r1, r2), outs):
        assert gb.lib.bddc_apply(pre._handle, gb._ptr(r), gb._ptr(want), stream) == 0
        assert gb.lib.bddc_apply_noalloc(pre._handle, gb._ptr(r), gb._ptr(got), stream) == 0
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - w).max() <= tol * np.abs(w).max()
    assert torch.cuda.mem_get_info()[0] == free_before
    pre.close()


def test_apply_noalloc_after_larger_problem():
    """A smaller problem after a larger one on the same device: stale contents
    of the shared array from the larger call must not leak into the result."""
    import paper_2001_07289_gb300.bddc as gb
    big = inputs.box_problem(24, 24, 24, [[12]] * 3, 4, alpha=inputs.alpha_loguniform(24, 24, 24, -1, 1, 2))
    small = inputs.box_problem(10, 9, 8, [[3, 7], [2, 5], [4]], 2, alpha=inputs.alpha_loguniform(10, 9, 8, -1, 1, 4))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pb = gb.BDDC.from_problem(big)
    rb = torch.from_numpy(inputs.random_node_vector(24, 24, 24, 5)).cuda()
    zb = torch.empty_like(rb)
    assert gb.lib.bddc_apply_noalloc(pb._handle, gb._ptr(rb), gb._ptr(zb), stream) == 0
    ps = gb.BDDC.from_problem(small)
    rs = torch.from_numpy(inputs.random_node_vector(10, 9, 8, 6)).cuda()
    want, got = torch.empty_like(rs), torch.empty_like(rs)
    assert gb.lib.bddc_apply(ps._handle, gb._ptr(rs), gb._ptr(want), stream) == 0
    assert gb.lib.bddc_apply_noalloc(ps._handle, gb._ptr(rs), gb._ptr(got), stream) == 0
    torch.cuda.synchronize()
    w, g = want.cpu().numpy(), got.cpu().numpy()
    assert np.abs(g - w).max() <= 1e-10 * np.abs(w).max()
    pb.close()
    ps.close()


def test_apply_noalloc_rejects_a_problem_above_the_limit():
    """A problem whose apply needs more work space than the fixed array holds
    (112^3 nodes on the mixed path, about 36 MB against 32 MiB) is refused
    with BDDC_ERR_ARG and a message giving the bytes needed; nothing is
    launched, so the output vector is left as it was."""
    import re
    import paper_2001_07289_gb300.bddc as gb
    n = 112
    p = inputs.box_problem(n, n, n, [inputs.uniform_cuts(n, 8)] * 3, 4, precision="mixed")
    pre = gb.BDDC.from_problem(p)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    r = torch.from_numpy(inputs.random_node_vector(n, n, n, 7)).cuda()
    z = torch.full_like(r, 5.0)
    code = gb.lib.bddc_apply_noalloc(pre._handle, gb._ptr(r), gb._ptr(z), stream)
    assert code == gb.BDDC_ERR_ARG
    msg = gb.lib.bddc_last_error(pre._handle).decode()
    need = int(re.search(r"needs (\d+) bytes", msg).group(1))
    assert need > (32 << 20)
    torch.cuda.synchronize()
    assert torch.all(z == 5.0)
    pre.close()
