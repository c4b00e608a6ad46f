"""GPU parity of the objective and its pieces against the FP64 oracle.

Every call goes through the C ABI of libreg.so (ctypes binding); inputs are
seeded and synthetic; the oracle receives the same FP32 values in FP64.
"""
import numpy as np
import pytest

from synth import make_pair, random_image, random_field
from tests.helpers import (J_RTOL, GRAD_RTOL, assert_parity, check_directional_fd, compare_eval, default_nodes,
                           full_size_node_bound, fused_seam_nodes, fused_tile_columns, rel_l2)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def reg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06765_gb300 as reg
    return reg


# 0: fused pass (ratio-2 grids); 1: multi-pass with the gather P^T of Eq. 3;
# A/B baselines of P^T: 2 atomic scatter, 3 8-colour scatter (ratio-2 levels)
EVAL_IMPLS = [0, 1, 2, 3]

# (dims, spacing, nodes or None, tau, rho, alpha, amplitude of u in mm)
CASES = [
    ((30, 26, 22), (1.0, 1.0, 1.0), None, 0.05, 0.05, 1.0, 1.5),          # ragged tiles (28 x 28 output)
    ((58, 38, 70), (1.2, 0.8, 1.0), None, 0.05, 0.03, 2.0, 2.5),          # several tiles and z segments
    ((28, 12, 8), (1.0, 1.0, 1.0), None, 0.1, 0.1, 1.0, 0.8),             # one tile, ragged in y
    ((28, 28, 8), (1.0, 1.0, 1.0), None, 0.1, 0.1, 1.0, 0.8),             # exactly one tile
    ((86, 58, 12), (1.0, 1.0, 1.0), None, 0.05, 0.05, 1.0, 1.5),          # 4 x 3 tiles, one thin column
    ((4, 6, 4), (1.0, 1.0, 1.0), None, 0.1, 0.1, 1.0, 0.3),               # smallest even grid
    ((16, 16, 16), (1.0, 1.0, 1.0), None, 0.05, 0.05, 1.0, 1.0),          # one tile
    ((37, 29, 23), (1.0, 1.1, 0.9), None, 0.05, 0.02, 3.0, 1.5),          # ragged, non-integer ratio
    ((40, 36, 20), (0.97, 0.97, 2.5), None, 0.1, 0.1, 50.0, 3.0),         # anisotropic spacing
    ((33, 48, 17), (1.5, 1.5, 1.5), ((9, 13, 5),), 0.08, 0.08, 5.0, 2.0),  # explicit node dims (ratio ~4)
    ((8, 6, 5), (1.0, 1.0, 1.0), None, 0.1, 0.1, 1.0, 0.5),               # tiny
    ((64, 64, 64), (1.0, 1.0, 1.0), None, 0.01, 0.01, 10.0, 2.0),         # 64^3 workload shape
]


@pytest.mark.parametrize("impl", EVAL_IMPLS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_eval_parity(reg_mod, orc, impl, case):
    dims, h, nodes, tau, rho, alpha, amp = CASES[case]
    R = random_image(dims, 100 + case)
    T = random_image(dims, 200 + case)
    cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, node_dims=nodes, eval_impl=impl)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    info = r.level_info(0)
    assert info["nodes"] == (nodes[0] if nodes else default_nodes(dims))
    u = random_field(info["nodes"], 300 + case, amp)
    e = compare_eval(r, orc, R, T, dims, h, u, tau, rho, alpha)
    assert e["eD"] <= J_RTOL, e
    assert e["eS"] <= 1e-5, e
    assert_parity(e)
    r.close()


@pytest.mark.parametrize("case", [c for c in range(len(CASES)) if CASES[c][2] is None])
def test_curvature_in_fused_pass_parity(reg_mod, orc, case):
    # fused_tz = -1: the fused pass forms the curvature Laplacian w and one S
    # partial per tile itself (the batched arithmetic); every node of w and S
    # must be formed by exactly one tile, ragged tiles and z segments included
    dims, h, nodes, tau, rho, alpha, amp = CASES[case]
    R = random_image(dims, 100 + case)
    T = random_image(dims, 200 + case)
    cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, fused_tz=-1)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    u = random_field(r.level_info(0)["nodes"], 300 + case, amp)
    e = compare_eval(r, orc, R, T, dims, h, u, tau, rho, alpha)
    assert e["eD"] <= J_RTOL, e
    assert e["eS"] <= 1e-5, e
    assert_parity(e)
    r.close()


@pytest.mark.parametrize("seams_only", [False, True])
def test_curvature_in_fused_pass_z_segments(reg_mod, orc, seams_only):
    # 300 planes: the throughput rule cuts segments of 64, 64, 64, 64 and 44
    # planes, which share the node planes 32, 64, 96 and 128; with seams_only
    # u is non-zero only there and on the node columns and rows that x and y
    # tiles share, so a seam node formed twice or never shows in S and grad
    dims, h, tau, rho, alpha = (30, 26, 300), (1.0, 1.2, 0.9), 0.05, 0.05, 4.0
    R = random_image(dims, 181)
    T = random_image(dims, 182)
    cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, fused_tz=-1)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    z, tiles = r.level_tiling(0)
    ntx, nty = fused_tile_columns(dims)
    assert z == 64 and tiles == ntx * nty * 5
    nodes = r.level_info(0)["nodes"]
    u = random_field(nodes, 183, 2.0)
    if seams_only:
        keep = np.zeros(u.shape[1:], bool)
        keep[:, :, fused_seam_nodes(dims[0], 0)] = True
        keep[:, fused_seam_nodes(dims[1], 1), :] = True
        keep[[32, 64, 96, 128], :, :] = True
        u = np.where(keep[None], u, 0.0).astype(np.float32)
    e = compare_eval(r, orc, R, T, dims, h, u, tau, rho, alpha)
    assert e["eS"] <= 1e-5, e
    assert_parity(e)
    r.close()


@pytest.mark.parametrize("impl", EVAL_IMPLS)
def test_eval_T_equals_R_is_zero(reg_mod, impl):
    dims, h = (30, 26, 22), (1.0, 1.0, 1.0)
    R = random_image(dims, 7)
    cfg = reg_mod.make_config(levels=1, tau=0.05, alpha=2.0, eval_impl=impl)
    r = reg_mod.Registration(cfg).set_images(R, R, h)
    u = torch.zeros(r.node_shape(0), device="cuda")
    J, D, S, g = r.eval(u)
    assert abs(D) < 1e-6 * R.size and S == 0.0
    assert float(g.abs().max()) < 1e-5
    r.close()


@pytest.mark.parametrize("impl", EVAL_IMPLS)
def test_eval_integer_shift_minimum(reg_mod, impl):
    # T_j = R_{j - s}; the constant displacement s h gives J = 0 (sign of x + P u)
    dims, h = (32, 28, 24), (1.0, 1.5, 2.0)
    s = (2, -1, 1)
    R = np.zeros(dims[::-1], np.float32)
    R[5:-5, 5:-5, 5:-5] = random_image((dims[0] - 10, dims[1] - 10, dims[2] - 10), 17)
    T = np.roll(R, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
    cfg = reg_mod.make_config(levels=1, tau=0.05, alpha=2.0, eval_impl=impl)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    shape = r.node_shape(0)
    u = torch.stack([torch.full(shape[1:], s[d] * h[d], device="cuda") for d in range(3)])
    J, D, S, g = r.eval(u)
    assert abs(J) < 1e-6 * R.size
    J2, *_ = r.eval(-u)
    assert J2 > 1.0
    r.close()


@pytest.mark.slow
@pytest.mark.parametrize("config_id", [2, 3])
def test_eval_parity_full_size(reg_mod, orc, config_id):
    """Full-size images (256^3 and 256x256x112) at a smooth random u: J and grad J."""
    from synth import CONFIGS
    p = make_pair(config_id)
    c = CONFIGS[config_id]
    cfg = reg_mod.make_config(levels=c["levels"], tau=c["eta"], alpha=c["alpha"])
    r = reg_mod.Registration(cfg).set_images(p["R"], p["T"], p["spacing"])
    info = r.level_info(0)
    u = random_field(info["nodes"], 400 + config_id, 5.0)
    e = compare_eval(r, orc, p["R"], p["T"], p["dims"], p["spacing"], u, c["eta"], c["eta"], c["alpha"])
    print({k: v for k, v in e.items() if k not in ("g", "go")})
    assert_parity(e, node_bound=False)
    full_size_node_bound(e)
    r.close()


def test_pyramid_parity(reg_mod, orc):
    dims, h = (37, 30, 23), (1.0, 1.0, 2.0)
    R = random_image(dims, 61, smooth=False)
    T = random_image(dims, 62, smooth=False)
    cfg = reg_mod.make_config(levels=3, tau=0.1)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    Ro, To, m = R.astype(np.float64), T.astype(np.float64), dims
    for lv in range(1, 3):
        Ro, To = orc.restrict(m, Ro), orc.restrict(m, To)
        m = tuple((v + 1) // 2 for v in m)
        info = r.level_info(lv)
        assert info["dims"] == m
        assert info["spacing"] == tuple(hh * 2 ** lv for hh in h)
        np.testing.assert_allclose(r.level_image(lv, "R").cpu().numpy(), Ro, rtol=0, atol=2e-6)
        np.testing.assert_allclose(r.level_image(lv, "T").cpu().numpy(), To, rtol=0, atol=2e-6)
    r.close()


def test_prolong_parity(reg_mod, orc):
    dims, h = (48, 40, 36), (1.0, 1.2, 1.5)
    R = random_image(dims, 71)
    cfg = reg_mod.make_config(levels=3, tau=0.1)
    r = reg_mod.Registration(cfg).set_images(R, R, h)
    for lc in (2, 1):
        ic, if_ = r.level_info(lc), r.level_info(lc - 1)
        uc = random_field(ic["nodes"], 72 + lc, 2.0)
        uf = r.prolong(torch.from_numpy(uc).cuda(), lc).cpu().numpy()
        ext_c = tuple(ic["dims"][d] * ic["spacing"][d] for d in range(3))
        ext_f = tuple(if_["dims"][d] * if_["spacing"][d] for d in range(3))
        ref = orc.prolong(ic["nodes"], ext_c, uc, if_["nodes"], ext_f)
        np.testing.assert_allclose(uf, ref, rtol=0, atol=2e-6)
    r.close()


@pytest.mark.parametrize("count", [0, 1, 3, 5])
def test_lbfgs_direction_parity(reg_mod, orc, count):
    dims, h = (16, 16, 16), (1.0, 1.0, 1.0)
    R = random_image(dims, 81)
    r = reg_mod.Registration(reg_mod.make_config(levels=1, mem=5)).set_images(R, R, h)
    n = 3 * 9 ** 3
    rng = np.random.default_rng(82 + count)
    A = rng.normal(size=(n, 8))
    # pairs of an SPD quadratic with a spread spectrum so that s'y > 0
    S = rng.normal(size=(count, n))
    Y = S * rng.uniform(0.5, 3.0, size=n) + 0.1 * (S @ A) @ A.T / n
    g = rng.normal(size=n)
    S32, Y32, g32 = (np.ascontiguousarray(a, np.float32) for a in (S, Y, g))
    p = r.lbfgs_direction(torch.from_numpy(S32).cuda() if count else None,
                          torch.from_numpy(Y32).cuda() if count else None,
                          torch.from_numpy(g32).cuda()).cpu().numpy()
    if count:
        gamma = float(S32[-1].astype(np.float64) @ Y32[-1]) / float(Y32[-1].astype(np.float64) @ Y32[-1])
        ref = -orc.two_loop(S32, Y32, g32, gamma)
    else:
        ref = -g32.astype(np.float64) * (1.0 / np.abs(g32).max())   # node spacing 1 on this grid
        ref *= min(r.level_info(0)["node_spacing"])
    assert rel_l2(p, ref) < 2e-5
    r.close()


def test_errors_are_reported(reg_mod):
    from paper_1812_06765_gb300 import _lib
    cfg = reg_mod.make_config(levels=1)
    r = reg_mod.Registration(cfg)
    u = torch.zeros(3 * 9 * 9 * 9, device="cuda")
    with pytest.raises(reg_mod.RegError) as ei:
        _lib.reg_eval_objective_grad(r.h, 0, u.data_ptr(), u.data_ptr())
    assert ei.value.code == _lib.REG_ERR_STATE
    with pytest.raises(reg_mod.RegError) as ei:
        r.set_images(np.zeros((3, 8, 8), np.float32), np.zeros((3, 8, 8), np.float32), (1, 1, 1))
    assert ei.value.code == _lib.REG_ERR_ARG
    with pytest.raises(reg_mod.RegError) as ei:
        r.set_images(np.zeros((8, 8, 8), np.float32), np.zeros((8, 8, 8), np.float32), (1, 0, 1))
    assert ei.value.code == _lib.REG_ERR_ARG
    r.set_images(random_image((16, 16, 16), 1), random_image((16, 16, 16), 2), (1, 1, 1))
    with pytest.raises(reg_mod.RegError):
        _lib.reg_eval_objective_grad(r.h, 3, u.data_ptr(), u.data_ptr())
    # a NaN image gives a numeric error, not a fault
    bad = random_image((16, 16, 16), 3)
    bad[4, 4, 4] = np.nan
    r.set_images(bad, bad, (1, 1, 1))
    with pytest.raises(reg_mod.RegError) as ei:
        r.eval(u)
    assert ei.value.code == _lib.REG_ERR_NUMERIC
    r.close()
    with pytest.raises(reg_mod.RegError):
        reg_mod.Registration(reg_mod.make_config(levels=0))


def test_autograd_function(reg_mod, orc):
    """RegObjective: backward = the hand-written adjoint gradient (= oracle gradient),
    and a directional finite difference of the forward agrees with the oracle's."""
    from paper_1812_06765_gb300 import RegObjective
    dims, h = (32, 28, 24), (1.0, 1.0, 1.0)
    R, T = random_image(dims, 91, noise=0.0), random_image(dims, 92, noise=0.0)
    tau, alpha = 0.05, 2.0
    r = reg_mod.Registration(reg_mod.make_config(levels=1, tau=tau, alpha=alpha)).set_images(R, T, h)
    nodes = r.level_info(0)["nodes"]
    u = torch.from_numpy(random_field(nodes, 93, 1.0)).cuda().requires_grad_(True)
    J = RegObjective.apply(u, r, 0)
    loss = 2.0 * J + (u.double() ** 2).sum()
    loss.backward()
    _, _, _, g = r.eval(u.detach())
    np.testing.assert_allclose(u.grad.cpu().numpy(), (2.0 * g + 2.0 * u.detach()).cpu().numpy(), rtol=1e-6,
                               atol=1e-6)
    u32 = u.detach().cpu().numpy()
    Jo, _, _, go = orc.objective(dims, h, R, T, nodes, u32, tau, tau, alpha)
    assert rel_l2(g.cpu().numpy(), go) <= GRAD_RTOL
    assert abs(J.item() - Jo) <= J_RTOL * abs(Jo)
    d = random_field(nodes, 94, 1.0)
    check_directional_fd(r, orc, 0, (dims, h, R, T, nodes, tau, alpha), u32, d, g.cpu().numpy())
    r.close()


@pytest.mark.parametrize("impl", [0, 1, "curv-in-pass"])
def test_seam_nodes_only_field(reg_mod, orc, impl):
    """u non-zero only on the node columns and rows that neighbouring tiles share
    along x and y and on the z node planes where segments of the split meet
    (20, 25, 30): the displacement jumps across every seam, so a seam node that a
    tile reads or gathers wrongly shows in the per-node bound."""
    dims, h, tau, rho, alpha = (58, 38, 70), (1.2, 0.8, 1.0), 0.05, 0.03, 2.0
    R = random_image(dims, 171)
    T = random_image(dims, 172)
    split = (40, 1, 10, 2, 10)
    if impl == "curv-in-pass":   # the throughput rule's uniform segments, curvature formed per tile
        cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, fused_tz=-1)
    else:
        cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, eval_impl=impl,
                                  fused_split=split if impl == 0 else None)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    nodes = r.level_info(0)["nodes"]
    if impl == 0:
        assert r.level_split(0) == split
    u = random_field(nodes, 173, 2.5)
    keep = np.zeros(u.shape[1:], bool)
    keep[:, :, fused_seam_nodes(dims[0], 0)] = True
    keep[:, fused_seam_nodes(dims[1], 1), :] = True
    keep[[20, 25, 30], :, :] = True
    u = np.where(keep[None], u, 0.0).astype(np.float32)
    e = compare_eval(r, orc, R, T, dims, h, u, tau, rho, alpha)
    assert_parity(e)
    r.close()


def _bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).bfloat16().float().numpy()


@pytest.mark.parametrize("config_id", [None, 2])
def test_bf16_image_storage(reg_mod, orc, config_id):
    """BF16 image storage, FP32 arithmetic: against the oracle fed the BF16-rounded
    images the kernel error meets the FP32 bar; against the FP32-image oracle the
    storage error is reported (and bounded loosely)."""
    from synth import CONFIGS
    if config_id is None:
        dims, h, tau, alpha = (58, 38, 70), (1.2, 0.8, 1.0), 0.05, 2.0
        R, T = random_image(dims, 601), random_image(dims, 602)
        amp, levels = 2.0, 1
    else:
        p = make_pair(config_id)
        c = CONFIGS[config_id]
        dims, h, tau, alpha, R, T = p["dims"], p["spacing"], c["eta"], c["alpha"], p["R"], p["T"]
        amp, levels = 5.0, c["levels"]
    cfg = reg_mod.make_config(levels=levels, tau=tau, alpha=alpha, image_dtype="bf16")
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    u = random_field(r.level_info(0)["nodes"], 603, amp)
    Rb, Tb = _bf16_round(R), _bf16_round(T)
    e_kernel = compare_eval(r, orc, Rb, Tb, dims, h, u, tau, tau, alpha)
    e_store = compare_eval(r, orc, R, T, dims, h, u, tau, tau, alpha)
    print("bf16 kernel error J %.2e grad %.2e; storage error J %.2e grad %.2e"
          % (e_kernel["eJ"], e_kernel["eg"], e_store["eJ"], e_store["eg"]))
    assert e_kernel["eJ"] <= J_RTOL and e_kernel["eg"] <= GRAD_RTOL, e_kernel
    assert e_store["eJ"] <= 1e-2 and e_store["eg"] <= 0.2, e_store
    r.close()


# z segment lengths: the throughput rule's powers of two, splits of the depth
# 70 into equal even segments (what the model and the autotuner pick from),
# ragged last segments, segments as long as or longer than the image
TZ_LENGTHS = [2, 4, 6, 10, 16, 24, 36, 70, 72, 128]


@pytest.mark.parametrize("tz", TZ_LENGTHS)
def test_every_fused_tile_depth_matches_oracle(reg_mod, orc, tz):
    # tiles sharing node planes in z, a forced segment length on every level
    dims, h, tau, rho, alpha = (58, 38, 70), (1.2, 0.8, 1.0), 0.05, 0.03, 2.0
    R = random_image(dims, 71)
    T = random_image(dims, 72)
    cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, fused_tz=tz)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    z, tiles = r.level_tiling(0)
    ntx, nty = fused_tile_columns(dims)
    assert z == min(tz, dims[2]) and tiles == ntx * nty * -(-dims[2] // tz)
    u = random_field(r.level_info(0)["nodes"], 73, 2.5)
    e = compare_eval(r, orc, R, T, dims, h, u, tau, rho, alpha)
    assert_parity(e)
    r.close()


# z splits of the depth 70 into segments of different lengths (l1, n1, l2, n2, lr):
# longest first in launch order, a short remainder, two groups without a
# remainder, the remainder longest
SPLITS = [(40, 1, 10, 2, 10), (30, 1, 20, 2, 0), (4, 2, 6, 3, 44), (16, 2, 2, 1, 36)]


@pytest.mark.parametrize("split", SPLITS)
def test_uneven_z_splits_match_oracle(reg_mod, orc, split):
    # tiles of unequal segments share node planes in z; the gather finds each
    # node plane's segment and the previous segment's last plane
    dims, h, tau, rho, alpha = (58, 38, 70), (1.2, 0.8, 1.0), 0.05, 0.03, 2.0
    R = random_image(dims, 71)
    T = random_image(dims, 72)
    cfg = reg_mod.make_config(levels=1, tau=tau, rho=rho, alpha=alpha, fused_split=split)
    r = reg_mod.Registration(cfg).set_images(R, T, h)
    l1, n1, l2, n2, lr = split
    assert r.level_split(0) == split
    z, tiles = r.level_tiling(0)
    ntx, nty = fused_tile_columns(dims)
    assert z == max(l1 if n1 else 0, l2 if n2 else 0, lr) and tiles == ntx * nty * (n1 + n2 + (lr > 0))
    u = random_field(r.level_info(0)["nodes"], 73, 2.5)
    e = compare_eval(r, orc, R, T, dims, h, u, tau, rho, alpha)
    assert_parity(e)
    r.close()


def test_autotuned_tiling_is_cached_per_geometry(reg_mod):
    dims, h = (96, 80, 64), (1.0, 1.0, 1.0)
    R = random_image(dims, 81)
    cfg = reg_mod.make_config(levels=3, tau=0.05, alpha=1.0)
    r1 = reg_mod.Registration(cfg).set_images(R, R, h)
    r2 = reg_mod.Registration(cfg).set_images(R, R, h)
    for lv in range(3):   # longest segment of the chosen split, and the tiles
        t1, t2 = r1.level_tiling(lv), r2.level_tiling(lv)
        depth = r1.level_info(lv)["dims"][2]
        assert t1 == t2 and t1[0] % 2 == 0 and 2 <= t1[0] <= depth and t1[1] > 0
    off = reg_mod.Registration(reg_mod.make_config(levels=3, tau=0.05, alpha=1.0, autotune=False))
    off.set_images(R, R, h)
    for lv in range(3):   # the load model's choice
        tz, tiles = off.level_tiling(lv)
        assert tz % 2 == 0 and 2 <= tz <= off.level_info(lv)["dims"][2] and tiles > 0
    for r in (r1, r2, off):
        r.close()


def test_ngf_pass_timing_query(reg_mod):
    from paper_1812_06765_gb300 import _lib
    dims = (64, 48, 40)
    R = random_image(dims, 91)
    r = reg_mod.Registration(reg_mod.make_config(levels=1, tau=0.05)).set_images(R, R, (1.0, 1.0, 1.0))
    with pytest.raises(_lib.RegError) as ei:
        _lib.reg_last_ngf_ms(r.h)
    assert ei.value.code == _lib.REG_ERR_STATE
    u = torch.zeros(r.node_shape(0), device="cuda")
    r.eval(u)
    ms = _lib.reg_last_ngf_ms(r.h)
    assert 0.0 < ms < 1000.0
    r.close()
