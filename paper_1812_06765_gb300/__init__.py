"""GB300-native matrix-free NGF + curvature deformable 3D image registration.

Budelmann, Koenig, Papenberg, Lellmann, "Fully-deformable 3D image
registration in two seconds" (BVM 2019): minimise
J(y) = D_NGF(R, T(P y)) + alpha S_curv(y) (Sec. 2.1, Eq. 1) with L-BFGS in a
coarse-to-fine pyramid, the objective and its gradient evaluated matrix-free
(Sec. 2.2, Eq. 2-3).

All computation runs in the CUDA library libreg.so (C ABI, include/reg.h);
this package marshals arguments and uses PyTorch only for device memory and
streams.  Arrays: images (m_z, m_y, m_x) float32; displacements
(3, n_z, n_y, n_x) float32 in mm (component planes x, y, z).
"""
import numpy as np
import torch

from . import _lib
from ._lib import RegConfig, RegError, RegStats  # noqa: F401

__all__ = ["make_config", "Registration", "RegObjective", "register", "register_batch", "RegError"]


def make_config(levels=1, tau=0.01, rho=None, alpha=10.0, mem=5, max_iter=50, c1=1e-4, max_backtracks=20,
                tol_grad_rel=1e-5, tol_j_rel=1e-7, tol_j_count=3, fixed_iters=False, start_level=-1,
                node_dims=None, eval_impl=None, use_graph=None, image_dtype=None, autotune=None, fused_tz=None,
                fused_split=None):
    """A reg_config; max_iter is one value for every level or a per-level list (index 0 = finest).
    image_dtype: "f32" (default) or "bf16" (the fused pass reads BF16 copies of the images).
    autotune: time the fused pass's z splits per level (default on); fused_tz: force equal segments
    of that length; fused_split: force (l1, n1, l2, n2, lr) on levels of that depth."""
    cfg = _lib.reg_config_default()
    cfg.tau = float(tau)
    cfg.rho = float(tau if rho is None else rho)
    cfg.alpha = float(alpha)
    cfg.c1 = float(c1)
    cfg.max_backtracks = int(max_backtracks)
    cfg.tol_grad_rel = float(tol_grad_rel)
    cfg.tol_j_rel = float(tol_j_rel)
    cfg.tol_j_count = int(tol_j_count)
    cfg.levels = int(levels)
    cfg.lbfgs_mem = int(mem)
    cfg.fixed_iters = int(bool(fixed_iters))
    cfg.start_level = int(start_level)
    its = list(max_iter) if hasattr(max_iter, "__len__") else [max_iter] * _lib.MAX_LEVELS
    for lv in range(_lib.MAX_LEVELS):
        cfg.max_iter[lv] = int(its[lv] if lv < len(its) else its[-1])
        for d in range(3):
            cfg.node_dims[lv][d] = 0 if node_dims is None or lv >= len(node_dims) else int(node_dims[lv][d])
    if eval_impl is not None:
        cfg.eval_impl = int(eval_impl)
    if use_graph is not None:
        cfg.use_graph = int(bool(use_graph))
    if image_dtype is not None:
        if image_dtype not in ("f32", "bf16"):
            raise ValueError("image_dtype must be 'f32' or 'bf16'")
        cfg.image_dtype = 1 if image_dtype == "bf16" else 0
    if autotune is not None:
        cfg.autotune = int(bool(autotune))
    if fused_tz is not None:
        cfg.fused_tz = int(fused_tz)
    if fused_split is not None:
        for i, v in enumerate(fused_split):
            cfg.fused_split[i] = int(v)
    return cfg


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1812_06765_gb300 needs a CUDA GPU; there is no CPU path")


class Registration:
    """One handle of the C library: images, pyramid, evaluation and registration."""

    def __init__(self, cfg=None, stream=None, **kw):
        _require_cuda()
        self.cfg = cfg if cfg is not None else make_config(**kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = _lib.reg_create(self.cfg, self.stream.cuda_stream)
        self.dims = None

    # -- images -------------------------------------------------------------
    def set_images(self, R, T, spacing):
        """R, T: (m_z, m_y, m_x) float32 numpy arrays or torch tensors (host or CUDA)."""
        if isinstance(R, torch.Tensor):
            dev = R.is_cuda
            R = R.detach().to(torch.float32).contiguous()
            T = T.detach().to(device=R.device, dtype=torch.float32).contiguous()
            pr, pt = R.data_ptr(), T.data_ptr()
            if not dev:
                R, T = R.numpy(), T.numpy()
        else:
            dev = False
            R = np.ascontiguousarray(R, dtype=np.float32)
            T = np.ascontiguousarray(T, dtype=np.float32)
            pr, pt = R.ctypes.data, T.ctypes.data
        if tuple(R.shape) != tuple(T.shape) or len(R.shape) != 3:
            raise ValueError("R and T must be 3D arrays of equal shape")
        mz, my, mx = R.shape
        self.dims = (mx, my, mz)
        _lib.reg_set_images(self.h, pr, pt, self.dims, spacing, dev)
        self._keep = (R, T)  # device copies are taken on the handle's stream
        return self

    def level_info(self, level=0):
        m, n, h, H = _lib.reg_level_info(self.h, level)
        return dict(dims=m, nodes=n, spacing=h, node_spacing=H)

    def level_tiling(self, level=0):
        """(longest z segment, CTAs) of the fused pass on a level; (0, 0) for multi-pass levels."""
        return _lib.reg_level_tiling(self.h, level)

    def level_split(self, level=0):
        """(l1, n1, l2, n2, lr): the fused pass's z segments on a level; zeros for multi-pass levels."""
        return _lib.reg_level_split(self.h, level)

    def node_shape(self, level=0):
        n = self.level_info(level)["nodes"]
        return (3, n[2], n[1], n[0])

    def level_image(self, level, which="R"):
        m = self.level_info(level)["dims"]
        out = torch.empty((m[2], m[1], m[0]), dtype=torch.float32, device="cuda")
        _lib.reg_get_level_image(self.h, level, 0 if which == "R" else 1, out.data_ptr(), True)
        return out

    # -- objective ----------------------------------------------------------
    def eval(self, u, level=0, grad=None):
        """J, D, S and grad_u J at displacement u (CUDA tensor of node_shape(level))."""
        u = self._node_tensor(u, level)
        if grad is None:
            grad = torch.empty_like(u)
        J, D, S = _lib.reg_eval_objective_grad(self.h, level, u.data_ptr(), grad.data_ptr())
        return J, D, S, grad

    def prolong(self, uc, level_coarse):
        uc = self._node_tensor(uc, level_coarse)
        uf = torch.empty(self.node_shape(level_coarse - 1), dtype=torch.float32, device="cuda")
        _lib.reg_prolong(self.h, level_coarse, uc.data_ptr(), uf.data_ptr())
        return uf

    def lbfgs_direction(self, S, Y, g):
        """p = -H g for pairs S[j], Y[j] (CUDA tensors (count, n)), oldest first."""
        g = g.contiguous()
        p = torch.empty_like(g)
        count = 0 if S is None else int(S.shape[0])
        sp = S.contiguous().data_ptr() if count else 0
        yp = Y.contiguous().data_ptr() if count else 0
        _lib.reg_lbfgs_direction(self.h, g.numel(), count, sp, yp, g.data_ptr(), p.data_ptr())
        return p

    # -- registration -------------------------------------------------------
    def register(self, u_init=None, out="torch"):
        """Run the multilevel registration; returns (u on the finest nodes, stats dict).
        out: "torch" (CUDA tensor), "pinned" (page-locked host tensor) or "numpy"."""
        if out not in _OUTS:
            raise ValueError("out must be 'torch', 'pinned' or 'numpy'")
        u = _output_array(self.node_shape(0), out)
        iptr = None
        if u_init is not None:   # the start level's field, in the memory kind of the output
            if isinstance(u_init, torch.Tensor):
                u_init = u_init.detach()
            if out == "numpy":
                if isinstance(u_init, torch.Tensor):
                    u_init = u_init.cpu().numpy()
                u_init = np.ascontiguousarray(u_init, dtype=np.float32)
                iptr = u_init.ctypes.data
            else:
                u_init = torch.as_tensor(u_init, dtype=torch.float32)
                u_init = (u_init.to("cuda") if out == "torch" else u_init.cpu().pin_memory()).contiguous()
                iptr = u_init.data_ptr()
        uptr = u.ctypes.data if out == "numpy" else u.data_ptr()
        rc, st = _lib.reg_register(self.h, uptr, out == "torch", iptr)
        return u, _stats_dict(rc, st)

    def _node_tensor(self, u, level):
        shape = self.node_shape(level)
        if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float32):
            raise TypeError("u must be a float32 CUDA tensor")
        if tuple(u.shape) != shape and u.numel() != int(np.prod(shape)):
            raise ValueError("u has %s elements, level %d needs %s" % (tuple(u.shape), level, shape))
        return u.contiguous()

    def close(self):
        if getattr(self, "h", None):
            _lib.reg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RegObjective(torch.autograd.Function):
    """J(u) as a differentiable scalar: forward runs the objective kernels,
    backward returns grad_output * grad_u J from the same (hand-written
    adjoint) kernels; torch autograd is not involved in the gradient itself."""

    @staticmethod
    def forward(ctx, u, reg, level=0):
        J, D, S, grad = reg.eval(u.detach(), level)
        ctx.save_for_backward(grad)
        return torch.tensor(J, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (gJ.to(grad.dtype) * grad).reshape(grad.shape), None, None


_OUTS = ("torch", "pinned", "numpy")


def _output_array(shape, out):
    """Result array of a registration: a CUDA tensor, a page-locked host tensor
    (the device-to-host copy runs at full speed) or a numpy array."""
    if out == "torch":
        return torch.empty(shape, dtype=torch.float32, device="cuda")
    if out == "pinned":
        return torch.empty(shape, dtype=torch.float32, pin_memory=True)
    return np.empty(shape, dtype=np.float32)


def _stats_dict(rc, st):
    L = st.levels
    return dict(status=rc, iters=list(st.iters)[:L], evals=list(st.evals)[:L], level_status=list(st.level_status)[:L],
                J=list(st.J)[:L], J_final=st.J_final, D_final=st.D_final, S_final=st.S_final, seconds=st.seconds,
                kernel_launches=st.kernel_launches, level_seconds=list(st.level_seconds)[:L],
                tiling=list(st.tiling)[:L])


def register_batch(regs, out="torch"):
    """Register the pairs of several Registration handles together (one graph
    launch per pyramid level for all of them); returns a list of (u, stats).
    out: "torch" (CUDA tensors), "pinned" (page-locked host tensors) or "numpy"."""
    if out not in _OUTS:
        raise ValueError("out must be 'torch', 'pinned' or 'numpy'")
    outs = [_output_array(r.node_shape(0), out) for r in regs]
    ptrs = [o.ctypes.data if out == "numpy" else o.data_ptr() for o in outs]
    rc, stats = _lib.reg_register_batch([r.h for r in regs], ptrs, out == "torch")
    return [(o, _stats_dict(rc, s)) for o, s in zip(outs, stats)]


def register(R, T, spacing, out="torch", u_init=None, **cfg_kw):
    """Convenience: one registration of (R, T); returns (u, stats)."""
    reg = Registration(make_config(**cfg_kw))
    try:
        reg.set_images(R, T, spacing)
        return reg.register(u_init=u_init, out=out)
    finally:
        reg.close()
