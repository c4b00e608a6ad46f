"""Shared helpers of the GPU tests (CUDA path vs the FP64 oracle)."""
import numpy as np

# per-evaluation tolerances against the FP64 oracle
J_RTOL = 1e-5       # relative error of J
GRAD_RTOL = 1e-4    # relative L2 error of grad J


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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
                eg=rel_l2(g.cpu().numpy(), go), g=g.cpu().numpy(), go=go)
