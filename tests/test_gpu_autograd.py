"""RegObjective (torch.autograd.Function) on the 128^3 CT workload, 3 levels.

The workload of 128^3 CT images at 1.5 mm with a 3-level pyramid (32^3, 64^3,
128^3; nodes 17^3, 33^3, 65^3) runs in the plain form and in the
autograd.Function form.  On every level the backward (the kernels' adjoint
gradient, Sec. 2.2) is compared with the FP64 oracle gradient and checked by
directional finite differences, and a descent loop driven through autograd
reproduces the plain form's values bit for bit.
"""
import numpy as np
import pytest

from synth import CONFIGS, make_pair, random_field
from tests.helpers import assert_parity, check_directional_fd, compare_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ct128():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06765_gb300 as reg
    c = CONFIGS[1]
    p = make_pair(1)
    r = reg.Registration(reg.make_config(levels=c["levels"], tau=c["eta"], alpha=c["alpha"]))
    r.set_images(p["R"], p["T"], p["spacing"])
    yield reg, r, c
    r.close()


def level_problem(r, c, lv):
    info = r.level_info(lv)
    R = r.level_image(lv, "R").cpu().numpy()
    T = r.level_image(lv, "T").cpu().numpy()
    return info["dims"], info["spacing"], R, T, info["nodes"], c["eta"], c["alpha"]


@pytest.mark.parametrize("lv", [2, 1, 0])
def test_backward_matches_oracle_and_finite_differences(ct128, orc, lv):
    reg, r, c = ct128
    from paper_1812_06765_gb300 import RegObjective
    problem = level_problem(r, c, lv)
    dims, h, R, T, nodes, eta, alpha = problem
    u0 = random_field(nodes, 1100 + lv, 4.0)
    u = torch.from_numpy(u0).cuda().requires_grad_(True)
    J = RegObjective.apply(u, r, lv)
    J.backward()
    g = u.grad.detach().cpu().numpy()
    # the backward is the plain form's gradient, and J its value
    Jp, _, _, gp = r.eval(u.detach(), lv)
    assert J.item() == Jp
    np.testing.assert_array_equal(g, gp.cpu().numpy())
    # against the FP64 oracle on the level's own images
    e = compare_eval(r, orc, R, T, dims, h, u0, eta, eta, alpha, level=lv)
    assert_parity(e)
    check_directional_fd(r, orc, lv, problem, u0, random_field(nodes, 1200 + lv, 1.0), g)


def test_descent_loop_through_autograd_equals_plain_form(ct128):
    """Ten normalised gradient steps of 0.05 node spacings on the finest level, once
    with the gradient from loss.backward() through RegObjective and once from the
    plain evaluation call: the same J and u at every step, bit for bit."""
    reg, r, c = ct128
    from paper_1812_06765_gb300 import RegObjective
    lv = 0
    nodes = r.level_info(lv)["nodes"]
    step = 0.05 * min(r.level_info(lv)["node_spacing"])
    ua = torch.zeros(r.node_shape(lv), device="cuda")
    up = ua.clone()
    Ja, Jp = [], []
    for _ in range(10):
        x = ua.clone().requires_grad_(True)
        J = RegObjective.apply(x, r, lv)
        J.backward()
        Ja.append(J.item())
        ga = x.grad
        ua = ua - step * ga / ga.abs().max()
        J2, _, _, gp = r.eval(up, lv)
        Jp.append(J2)
        up = up - step * gp / gp.abs().max()
    assert Ja == Jp
    assert torch.equal(ua, up)
    assert Ja[1] < Ja[0]    # a short step along -g lowers J
    assert nodes == (65, 65, 65)
