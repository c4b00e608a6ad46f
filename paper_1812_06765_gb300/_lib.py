"""ctypes binding of libreg.so with the names of include/reg.h.

Argument marshalling only: every step of the registration runs in the CUDA
library.  Importing this module loads the library and raises if it has not
been built; there is no CPU path.
"""
import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libreg.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "reg.h")

MAX_LEVELS = 8
MAX_MEM = 8
MAX_VOXELS = 2147483647   # voxels of an image, and 3 x nodes of a deformation grid
MAX_PLANES = 65535        # m_z of an image, n_z of a deformation grid

REG_OK = 0
REG_WARN_LINESEARCH = 1
REG_ERR_ARG = -1
REG_ERR_CUDA = -2
REG_ERR_OOM = -3
REG_ERR_STATE = -4
REG_ERR_NUMERIC = -5
REG_ERR_TIMEOUT = -6


class RegConfig(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("rho", ctypes.c_double), ("alpha", ctypes.c_double),
        ("c1", ctypes.c_double), ("tol_grad_rel", ctypes.c_double), ("tol_j_rel", ctypes.c_double),
        ("tol_j_count", ctypes.c_int), ("levels", ctypes.c_int), ("lbfgs_mem", ctypes.c_int),
        ("max_backtracks", ctypes.c_int), ("fixed_iters", ctypes.c_int), ("start_level", ctypes.c_int),
        ("max_iter", ctypes.c_int * MAX_LEVELS), ("node_dims", (ctypes.c_int * 3) * MAX_LEVELS),
        ("eval_impl", ctypes.c_int), ("use_graph", ctypes.c_int), ("image_dtype", ctypes.c_int),
        ("autotune", ctypes.c_int), ("fused_tz", ctypes.c_int), ("test_expire_wait", ctypes.c_int),
        ("fused_split", ctypes.c_int * 5), ("reserved", ctypes.c_int * 1),
    ]


class RegStats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int), ("iters", ctypes.c_int * MAX_LEVELS), ("evals", ctypes.c_int * MAX_LEVELS),
        ("level_status", ctypes.c_int * MAX_LEVELS), ("J", ctypes.c_double * MAX_LEVELS),
        ("J_final", ctypes.c_double), ("D_final", ctypes.c_double), ("S_final", ctypes.c_double),
        ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_longlong), ("status", ctypes.c_int),
        ("level_seconds", ctypes.c_double * MAX_LEVELS), ("tiling", ctypes.c_int * MAX_LEVELS),
    ]


class RegError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libreg error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """The loaded libreg.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libreg.so not built (run __graft_entry__.build() or "
                               "python paper_1812_06765_gb300/build.py): " + LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        L.reg_version.restype = ctypes.c_int
        L.reg_config_default.argtypes = [ctypes.POINTER(RegConfig)]
        L.reg_config_default.restype = None
        L.reg_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(RegConfig), vp]
        L.reg_set_images.argtypes = [vp, fp, fp, ip, dp, ctypes.c_int]
        L.reg_level_info.argtypes = [vp, ctypes.c_int, ip, ip, dp, dp]
        L.reg_level_tiling.argtypes = [vp, ctypes.c_int, ip, ip]
        L.reg_level_split.argtypes = [vp, ctypes.c_int, ip]
        L.reg_fused_split_plan.argtypes = [ip, ctypes.c_int, ip, dp]
        L.reg_fused_split_plan.restype = ctypes.c_int
        L.reg_fused_tile_shape.argtypes = [ip, ip, ip]
        L.reg_fused_tile_shape.restype = ctypes.c_int
        L.reg_axis_tables.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ip, fp, ip, ip, fp, ctypes.c_int, ip]
        L.reg_axis_tables.restype = ctypes.c_int
        L.reg_get_level_image.argtypes = [vp, ctypes.c_int, ctypes.c_int, fp, ctypes.c_int]
        L.reg_eval_objective_grad.argtypes = [vp, ctypes.c_int, fp, fp, dp, dp, dp]
        L.reg_prolong.argtypes = [vp, ctypes.c_int, fp, fp]
        L.reg_last_ngf_ms.argtypes = [vp, dp]
        L.reg_lbfgs_direction.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, fp, fp, fp, fp]
        L.reg_register.argtypes = [vp, fp, ctypes.c_int, fp, ctypes.POINTER(RegStats)]
        L.reg_destroy.argtypes = [vp]
        L.reg_last_error.argtypes = [vp]
        L.reg_last_error.restype = ctypes.c_char_p
        L.reg_eval_objective_grad_noalloc.argtypes = [fp, fp, ip, dp, fp, fp, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_double, fp, vp]
        L.reg_eval_objective_grad_noalloc.restype = ctypes.c_int
        L.reg_register_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(fp), ctypes.c_int,
                                         ctypes.POINTER(RegStats)]
        L.reg_register_batch.restype = ctypes.c_int
        for name in ("reg_create", "reg_set_images", "reg_level_info", "reg_level_tiling", "reg_level_split",
                     "reg_last_ngf_ms",
                     "reg_get_level_image",
                     "reg_eval_objective_grad", "reg_prolong", "reg_lbfgs_direction", "reg_register",
                     "reg_destroy"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def header_functions():
    """Names of the functions include/reg.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(reg_\w+)\s*\(", text, re.M)))


def check(handle, code):
    """Raise RegError for a negative status; return the (non-negative) status."""
    if code < 0:
        raise RegError(code, last_error(handle))
    return code


def last_error(handle):
    msg = lib().reg_last_error(handle)
    return msg.decode() if msg else ""


# --- thin wrappers with the C names --------------------------------------------------------
def reg_version():
    return lib().reg_version()


def reg_config_default():
    cfg = RegConfig()
    lib().reg_config_default(ctypes.byref(cfg))
    return cfg


def reg_create(cfg, stream=None):
    h = ctypes.c_void_p()
    rc = lib().reg_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(stream or 0))
    if rc < 0:
        raise RegError(rc, last_error(None))
    return h


def reg_set_images(h, R_ptr, T_ptr, dims, spacing, ptr_is_device):
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    s = (ctypes.c_double * 3)(*[float(v) for v in spacing])
    return check(h, lib().reg_set_images(h, ctypes.c_void_p(R_ptr), ctypes.c_void_p(T_ptr), d, s,
                                         int(bool(ptr_is_device))))


def reg_level_info(h, level):
    m, n = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    sp, H = (ctypes.c_double * 3)(), (ctypes.c_double * 3)()
    check(h, lib().reg_level_info(h, int(level), m, n, sp, H))
    return tuple(m), tuple(n), tuple(sp), tuple(H)


def reg_level_tiling(h, level):
    tz, tiles = ctypes.c_int(), ctypes.c_int()
    check(h, lib().reg_level_tiling(h, int(level), ctypes.byref(tz), ctypes.byref(tiles)))
    return tz.value, tiles.value


def reg_fused_split_plan(dims, num_sms):
    """(split (l1, n1, l2, n2, lr), modelled steps) of the load model; host only."""
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    v = (ctypes.c_int * 5)()
    steps = ctypes.c_double()
    check(None, lib().reg_fused_split_plan(d, int(num_sms), v, ctypes.byref(steps)))
    return tuple(v), steps.value


def reg_fused_tile_shape():
    """(output columns per tile along x, along y, resident CTAs per SM) of the fused pass; host only."""
    ox, oy, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(None, lib().reg_fused_tile_shape(ctypes.byref(ox), ctypes.byref(oy), ctypes.byref(k)))
    return ox.value, oy.value, k.value


def reg_axis_tables(m, h, n):
    """(k0, w1, first, cnt, w) of one axis as numpy arrays (w: n x max weights); host only."""
    import numpy as np
    need = ctypes.c_int()
    check(None, lib().reg_axis_tables(int(m), float(h), int(n), None, None, None, None, None, 0, ctypes.byref(need)))
    k0, first, cnt = (np.zeros(int(m), np.int32), np.zeros(int(n), np.int32), np.zeros(int(n), np.int32))
    w1, w = np.zeros(int(m), np.float32), np.zeros((int(n), need.value), np.float32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)   # noqa: E731
    check(None, lib().reg_axis_tables(int(m), float(h), int(n), ctypes.cast(ptr(k0), ctypes.POINTER(ctypes.c_int)),
                                      ptr(w1), ctypes.cast(ptr(first), ctypes.POINTER(ctypes.c_int)),
                                      ctypes.cast(ptr(cnt), ctypes.POINTER(ctypes.c_int)), ptr(w), need.value, None))
    return k0, w1, first, cnt, w


def reg_level_split(h, level):
    v = (ctypes.c_int * 5)()
    check(h, lib().reg_level_split(h, int(level), v))
    return tuple(v)


def reg_get_level_image(h, level, which, out_ptr, out_is_device):
    return check(h, lib().reg_get_level_image(h, int(level), int(which), ctypes.c_void_p(out_ptr),
                                              int(bool(out_is_device))))


def reg_eval_objective_grad(h, level, u_ptr, grad_ptr, want_scalars=True):
    J, D, S = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    if want_scalars:
        check(h, lib().reg_eval_objective_grad(h, int(level), ctypes.c_void_p(u_ptr), ctypes.c_void_p(grad_ptr),
                                               ctypes.byref(J), ctypes.byref(D), ctypes.byref(S)))
        return J.value, D.value, S.value
    check(h, lib().reg_eval_objective_grad(h, int(level), ctypes.c_void_p(u_ptr), ctypes.c_void_p(grad_ptr),
                                           None, None, None))
    return None


def reg_eval_objective_grad_noalloc(R_ptr, T_ptr, dims, spacing, u_ptr, grad_ptr, tau, rho, alpha, jds_ptr,
                                    stream=None):
    """The allocation-free evaluation (no handle); J, D, S land in the device array at jds_ptr."""
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    s = (ctypes.c_double * 3)(*[float(v) for v in spacing])
    return check(None, lib().reg_eval_objective_grad_noalloc(
        ctypes.c_void_p(R_ptr), ctypes.c_void_p(T_ptr), d, s, ctypes.c_void_p(u_ptr), ctypes.c_void_p(grad_ptr),
        float(tau), float(rho), float(alpha), ctypes.c_void_p(jds_ptr), ctypes.c_void_p(stream or 0)))


def reg_last_ngf_ms(h):
    ms = ctypes.c_double()
    check(h, lib().reg_last_ngf_ms(h, ctypes.byref(ms)))
    return ms.value


def reg_prolong(h, level_coarse, uc_ptr, uf_ptr):
    return check(h, lib().reg_prolong(h, int(level_coarse), ctypes.c_void_p(uc_ptr), ctypes.c_void_p(uf_ptr)))


def reg_lbfgs_direction(h, n, count, S_ptr, Y_ptr, g_ptr, p_ptr):
    return check(h, lib().reg_lbfgs_direction(h, int(n), int(count), ctypes.c_void_p(S_ptr or 0),
                                              ctypes.c_void_p(Y_ptr or 0), ctypes.c_void_p(g_ptr),
                                              ctypes.c_void_p(p_ptr)))


def reg_register(h, u_out_ptr, out_is_device, u_init_ptr=None):
    st = RegStats()
    rc = check(h, lib().reg_register(h, ctypes.c_void_p(u_out_ptr), int(bool(out_is_device)),
                                     ctypes.c_void_p(u_init_ptr or 0), ctypes.byref(st)))
    return rc, st


def reg_register_batch(handles, u_out_ptrs, out_is_device):
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    outs = (ctypes.c_void_p * n)(*u_out_ptrs)
    stats = (RegStats * n)()
    rc = lib().reg_register_batch(hs, n, outs, int(bool(out_is_device)), stats)
    if rc < 0:
        msg = last_error(None) or last_error(handles[0])
        raise RegError(rc, msg)
    return rc, list(stats)


def reg_destroy(h):
    return lib().reg_destroy(h)


def reg_last_error(h):
    return last_error(h)
