"""The allocation-free evaluation entry point against the handle-based one.

reg_eval_objective_grad_noalloc serves callers that may not allocate device
memory while they run: its working memory is a fixed array in the library's
device image.  These tests call it through the C ABI twice in a row, with
different displacements, and check each result against reg_eval_objective_grad
on a handle; they also check that sizes beyond the fixed capacity and
malformed sizes are refused before anything is launched.  The file is named
to be collected last.
"""
import numpy as np
import pytest

from synth import random_field, random_image
from tests.helpers import GRAD_RTOL, J_RTOL, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def reg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06765_gb300 as reg
    return reg


def _noalloc(lib, R, T, dims, h, u, tau, rho, alpha):
    grad = torch.empty_like(u)
    jds = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    lib.reg_eval_objective_grad_noalloc(R.data_ptr(), T.data_ptr(), dims, h, u.data_ptr(), grad.data_ptr(), tau, rho,
                                        alpha, jds.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return jds.cpu().numpy(), grad


def test_noalloc_matches_handle_evaluation_on_two_calls(reg_mod):
    from paper_1812_06765_gb300 import _lib
    dims, h = (60, 44, 38), (1.0, 1.2, 0.9)       # several tiles and z segments, ragged edges
    tau, rho, alpha = 0.05, 0.04, 3.0
    R, T = random_image(dims, 501), random_image(dims, 502)
    Rd, Td = torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda()
    r = reg_mod.Registration(reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha)).set_images(R, T, h)
    nodes = r.level_info(0)["nodes"]
    assert nodes == tuple(m // 2 + 1 for m in dims)
    for call, seed in enumerate((503, 504)):       # two calls in a row share the scratch array
        u = torch.from_numpy(random_field(nodes, seed, 1.5 + call)).cuda()
        jds, grad = _noalloc(_lib, Rd, Td, dims, h, u, tau, rho, alpha)
        J, D, S, g_ref = r.eval(u)
        assert abs(jds[0] - J) <= J_RTOL * abs(J), (call, jds, J)
        assert abs(jds[1] - D) <= J_RTOL * abs(D), (call, jds, D)
        assert abs(jds[2] - S) <= 1e-5 * abs(S), (call, jds, S)
        assert rel_l2(grad.cpu().numpy(), g_ref.cpu().numpy()) <= GRAD_RTOL, call
    r.close()


def test_noalloc_refuses_sizes_beyond_its_capacity(reg_mod):
    from paper_1812_06765_gb300 import _lib
    u = torch.zeros(16, device="cuda")
    img = torch.zeros(16, device="cuda")
    jds = torch.zeros(3, dtype=torch.float64, device="cuda")
    for dims in ((256, 256, 256), (64, 64, 63), (2, 64, 64)):
        with pytest.raises(_lib.RegError) as ei:
            _lib.reg_eval_objective_grad_noalloc(img.data_ptr(), img.data_ptr(), dims, (1.0, 1.0, 1.0), u.data_ptr(),
                                                 u.data_ptr(), 0.1, 0.1, 1.0, jds.data_ptr())
        assert ei.value.code == _lib.REG_ERR_ARG
        assert _lib.reg_last_error(None)
    # R is read two voxels at a time: a pointer 4 bytes off an 8-byte boundary is refused before any launch
    with pytest.raises(_lib.RegError) as ei:
        _lib.reg_eval_objective_grad_noalloc(img.data_ptr() + 4, img.data_ptr(), (32, 32, 32), (1.0, 1.0, 1.0),
                                             u.data_ptr(), u.data_ptr(), 0.1, 0.1, 1.0, jds.data_ptr())
    assert ei.value.code == _lib.REG_ERR_ARG and "aligned" in _lib.reg_last_error(None)
    assert float(jds.abs().sum()) == 0.0           # nothing was written
