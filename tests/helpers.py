"""Shared helpers of the GPU tests (CUDA path vs the FP64 oracle)."""
import numpy as np

# per-evaluation tolerances against the FP64 oracle
J_RTOL = 1e-5       # relative error of J
GRAD_RTOL = 1e-4    # relative L2 error of grad J
# worst node: |g_k - g_o,k| <= GRAD_NODE_RTOL max|g_o| at every node entry.  The L2
# gate alone would hide a few wrong nodes (a tile seam, a segment's first plane).
GRAD_NODE_RTOL = 1e-3


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fused_tile_columns(dims):
    """Tile columns of the fused pass over an image (x tiles, y tiles), from the library's tile shape."""
    from paper_1812_06765_gb300 import _lib
    ox, oy, _ = _lib.reg_fused_tile_shape()
    return -(-dims[0] // ox), -(-dims[1] // oy)


def fused_seam_nodes(extent, axis):
    """Node indices that neighbouring fused tiles share along x (axis 0) or y (axis 1)."""
    from paper_1812_06765_gb300 import _lib
    o = _lib.reg_fused_tile_shape()[axis]
    return list(range(o // 2, extent // 2, o // 2))


def default_nodes(dims):
    return tuple(int(m) // 2 + 1 for m in dims)


def compare_eval(reg, orc, R, T, dims, h, u_np, tau, rho, alpha, level=0):
    """Evaluate on the GPU (through the C ABI) and with the oracle; return errors."""
    import torch
    info = reg.level_info(level)
    nodes = info["nodes"]
    u = torch.from_numpy(np.ascontiguousarray(u_np, dtype=np.float32)).cuda()
    J, D, S, g = reg.eval(u, level)
    Jo, Do, So, go = orc.objective(dims, h, R, T, nodes, u.cpu().numpy(), tau, rho, alpha)
    return dict(J=J, Jo=Jo, D=D, Do=Do, S=S, So=So,
                eJ=abs(J - Jo) / max(abs(Jo), 1e-300),
                eD=abs(D - Do) / max(abs(Do), 1e-300),
                eS=abs(S - So) / max(abs(So), 1e-300) if So != 0 else abs(S),
                eg=rel_l2(g.cpu().numpy(), go), g=g.cpu().numpy(), go=go, **node_errors(g.cpu().numpy(), go))


def node_errors(g, go):
    """Per-node-entry errors of a gradient, relative to max|g_o|: the worst one
    (eg_max), the 99.99th percentile (eg_p9999) and how many exceed GRAD_NODE_RTOL."""
    d = np.abs(np.asarray(g, np.float64) - np.asarray(go, np.float64)).ravel()
    scale = max(float(np.abs(go).max()), 1e-300)
    return dict(eg_max=float(d.max()) / scale, eg_p9999=float(np.quantile(d, 0.9999)) / scale,
                n_bad=int((d > GRAD_NODE_RTOL * scale).sum()))


def assert_parity(e, node_bound=True):
    """The per-evaluation bar against the oracle: J to J_RTOL, grad J to GRAD_RTOL in
    relative L2 and, with node_bound, every node entry to GRAD_NODE_RTOL max|g_o|."""
    summary = {k: v for k, v in e.items() if k not in ("g", "go")}
    assert e["eJ"] <= J_RTOL, summary
    assert e["eg"] <= GRAD_RTOL, summary
    if node_bound:
        assert e["eg_max"] <= GRAD_NODE_RTOL, summary


def full_size_node_bound(e):
    """Per-node bound at full size.  An FP32 sample coordinate within ~1e-7 voxel of
    a cell face can round to the other cell than the FP64 one; that voxel's
    interpolant gradient then jumps by a second difference of T, and its 8 nodes
    move by up to a few percent of the largest node gradient.  At ~6e-7 such voxels
    per voxel a volume of 10-70 M voxels has tens of them, so the GRAD_NODE_RTOL
    bound holds for all but 0.01 % of the node entries, and the worst entry may
    exceed it by such a jump, up to 1e-2 max|g_o| (measured: at most 9.7e-4 on the
    512 x 512 x 257 pair, 6.4e-5 on 512 x 512 x 256, 3.9e-5 at 256^3)."""
    summary = {k: v for k, v in e.items() if k not in ("g", "go")}
    assert e["eg_p9999"] <= GRAD_NODE_RTOL, summary
    assert e["eg_max"] <= 1e-2, summary


def check_directional_fd(r, orc, level, problem, u, d, g, eps=5e-2):
    """Central difference of the forward, (J(u + eps d) - J(u - eps d)) / 2 eps, through
    RegObjective on the GPU, against the same difference quotient of the FP64 oracle
    and against the analytic directional derivative g . d.

    J is only piecewise smooth: the trilinear interpolant's gradient jumps at cell
    faces, and a step of eps mm moves ~eps / h of the samples across one, so the
    difference quotient of the exact objective differs from g . d by a kink term
    (measured here on the oracle: ~1e-3 relative at eps = 5e-2).  The GPU forward
    must reproduce the oracle's quotient to 2e-3 of |g . d| (FP32 J over 2 eps), and
    its distance from g . d may exceed the oracle's only by that much."""
    import torch
    from paper_1812_06765_gb300 import RegObjective
    dims, h, R, T, nodes, tau, alpha = problem
    ut, dt = torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda(), torch.from_numpy(d).cuda()
    with torch.no_grad():
        up, um = ut + eps * dt, ut - eps * dt
        Jp = RegObjective.apply(up, r, level).item()
        Jm = RegObjective.apply(um, r, level).item()
    fd = (Jp - Jm) / (2 * eps)
    Jpo = orc.objective(dims, h, R, T, nodes, up.cpu().numpy(), tau, tau, alpha)[0]
    Jmo = orc.objective(dims, h, R, T, nodes, um.cpu().numpy(), tau, tau, alpha)[0]
    fdo = (Jpo - Jmo) / (2 * eps)
    an = float(np.sum(np.asarray(g, np.float64) * d))
    kink = abs(fdo - an)
    info = dict(fd=fd, fd_oracle=fdo, analytic=an, oracle_kink_rel=kink / abs(an))
    print(info)
    assert abs(fd - fdo) <= 2e-3 * abs(an), info
    assert abs(fd - an) <= kink + 2e-3 * abs(an), info
