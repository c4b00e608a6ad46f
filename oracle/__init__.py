"""FP64 CPU oracle (ctypes loader for ``reg_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The tests, the package's smoke check and the
benchmark's CPU-baseline leg are the only callers; the CUDA path never imports
this package and shares no code with it.

Arrays follow the C side: images are (m_z, m_y, m_x) float64 (x fastest),
displacements are (3, n_z, n_y, n_x) float64 planes, dims are (x, y, z) tuples.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 8


def build(force=False):
    """Compile the oracle with gcc (FP64, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC, os.path.join(_HERE, "reg_oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wno-unused-result",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Config(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("rho", ctypes.c_double), ("alpha", ctypes.c_double),
        ("c1", ctypes.c_double), ("tol_grad_rel", ctypes.c_double), ("tol_j_rel", ctypes.c_double),
        ("tol_j_count", ctypes.c_int), ("levels", ctypes.c_int), ("mem", ctypes.c_int),
        ("max_backtracks", ctypes.c_int), ("fixed_iters", ctypes.c_int), ("start_level", ctypes.c_int),
        ("max_iter", ctypes.c_int * MAX_LEVELS), ("node_dims", (ctypes.c_int * 3) * MAX_LEVELS),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int * MAX_LEVELS), ("evals", ctypes.c_int * MAX_LEVELS),
        ("status", ctypes.c_int * MAX_LEVELS), ("J", ctypes.c_double * MAX_LEVELS),
        ("D", ctypes.c_double * MAX_LEVELS), ("S", ctypes.c_double * MAX_LEVELS),
        ("mn", (ctypes.c_int * 3) * MAX_LEVELS), ("m", (ctypes.c_int * 3) * MAX_LEVELS),
    ]


# double fn(void *ctx, const double *u, double *g)
EVAL_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L = _lib
            L.orc_P.argtypes = [ip, dp, ip, dp, dp]
            L.orc_PT.argtypes = [ip, dp, ip, dp, dp]
            L.orc_PT_table.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int]
            L.orc_PT_table.restype = ctypes.c_int
            L.orc_interp.argtypes = [ip, dp, dp, ctypes.c_size_t, dp, dp, dp]
            L.orc_ngf.argtypes = [ip, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
            L.orc_ngf.restype = ctypes.c_double
            L.orc_ngf_adjoint.argtypes = [ip, dp, dp, dp]
            L.orc_curvature.argtypes = [ip, dp, dp, dp]
            L.orc_curvature.restype = ctypes.c_double
            L.orc_objective.argtypes = [ip, dp, dp, dp, ip, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, dp, dp, dp, dp]
            L.orc_restrict.argtypes = [ip, dp, dp]
            L.orc_prolong.argtypes = [ip, dp, dp, ip, dp, dp]
            L.orc_two_loop.argtypes = [ctypes.c_size_t, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp]
            L.orc_register.argtypes = [ip, dp, dp, dp, ctypes.POINTER(Config), dp, dp, ctypes.POINTER(Stats)]
            L.orc_register.restype = ctypes.c_int
            L.orc_lbfgs_level.argtypes = [ip, dp, dp, dp, ip, ctypes.POINTER(Config), ctypes.c_int, dp,
                                          ip, ip, dp]
            L.orc_lbfgs_level.restype = ctypes.c_int
            L.orc_lbfgs.argtypes = [ctypes.c_size_t, EVAL_FN, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.POINTER(Config), ctypes.c_int, dp, ip, ip, dp]
            L.orc_lbfgs.restype = ctypes.c_int
            L.orc_level_dims.argtypes = [ip, ctypes.POINTER(Config), ctypes.c_int, ip, ip]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_compensated_sums.argtypes = [ctypes.c_int]
            L.orc_set_compensated_sums.restype = None
            L.orc_sum.argtypes = [ctypes.c_size_t, dp]
            L.orc_sum.restype = ctypes.c_double
    return _lib


def _i3(v):
    return (ctypes.c_int * 3)(*[int(a) for a in v])


def _d3(v):
    return (ctypes.c_double * 3)(*[float(a) for a in v])


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return lib().orc_num_threads()


def set_compensated_sums(on):
    """Compensated (Neumaier) summation in every reduction of the oracle (default off:
    the plain running sum; both add the terms in index order)."""
    lib().orc_set_compensated_sums(int(bool(on)))


def reduce_sum(a):
    """The oracle's reduction of a 1-D array (plain or compensated, as set)."""
    a = _f64(np.ravel(a))
    return lib().orc_sum(a.size, _dp(a))


def node_spacing(dims, spacing, nodes):
    return tuple(dims[d] * spacing[d] / (nodes[d] - 1) for d in range(3))


def default_nodes(dims):
    """Node count rule m_d/2 + 1 per dimension."""
    return tuple(int(m) // 2 + 1 for m in dims)


def P(dims, spacing, nodes, u):
    """Grid conversion of one component u (n_z, n_y, n_x) -> (m_z, m_y, m_x)."""
    u = _f64(u)
    out = np.empty((dims[2], dims[1], dims[0]))
    lib().orc_P(_i3(dims), _d3(spacing), _i3(nodes), _dp(u), _dp(out))
    return out


def PT(dims, spacing, nodes, r):
    """Transpose of the grid conversion for one component (Eq. 3 gather)."""
    r = _f64(r)
    out = np.empty((nodes[2], nodes[1], nodes[0]))
    lib().orc_PT(_i3(dims), _d3(spacing), _i3(nodes), _dp(r), _dp(out))
    return out


def PT_table(m, h, mn, k, max_w=64):
    first = ctypes.c_int(0)
    w = np.zeros(max_w)
    cnt = lib().orc_PT_table(int(m), float(h), int(mn), int(k), ctypes.byref(first), _dp(w), max_w)
    return first.value, w[:cnt].copy()


def interp(dims, spacing, T, points):
    """Trilinear interpolation of T at points (N, 3) in mm -> (values, gradients (N, 3))."""
    T = _f64(T)
    pts = _f64(np.asarray(points, dtype=np.float64).T)
    n = pts.shape[1]
    val = np.empty(n)
    grad = np.empty((3, n))
    lib().orc_interp(_i3(dims), _d3(spacing), _dp(T), n, _dp(pts), _dp(val), _dp(grad))
    return val, grad.T.copy()


def ngf(dims, spacing, Tw, R, tau, rho):
    """NGF distance D (Eq. 2) of a deformed template and v = dpsi/da (3 planes)."""
    Tw, R = _f64(Tw), _f64(R)
    v = np.empty((3, dims[2], dims[1], dims[0]))
    D = lib().orc_ngf(_i3(dims), _d3(spacing), _dp(Tw), _dp(R), float(tau), float(rho), _dp(v))
    return D, v


def ngf_adjoint(dims, spacing, v):
    v = _f64(v)
    g = np.empty((dims[2], dims[1], dims[0]))
    lib().orc_ngf_adjoint(_i3(dims), _d3(spacing), _dp(v), _dp(g))
    return g


def curvature(nodes, H, u):
    """S and grad S for a displacement (3, n_z, n_y, n_x)."""
    u = _f64(u)
    g = np.empty_like(u)
    S = lib().orc_curvature(_i3(nodes), _d3(H), _dp(u), _dp(g))
    return S, g


def objective(dims, spacing, R, T, nodes, u, tau, rho, alpha):
    """J, D, S and grad_u J (3, n_z, n_y, n_x) in FP64."""
    R, T, u = _f64(R), _f64(T), _f64(u)
    grad = np.empty_like(u)
    J, D, S = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_objective(_i3(dims), _d3(spacing), _dp(R), _dp(T), _i3(nodes), _dp(u), float(tau), float(rho),
                        float(alpha), ctypes.byref(J), ctypes.byref(D), ctypes.byref(S), _dp(grad))
    return J.value, D.value, S.value, grad


def restrict(dims, img):
    img = _f64(img)
    mo = tuple((m + 1) // 2 for m in dims)
    out = np.empty((mo[2], mo[1], mo[0]))
    lib().orc_restrict(_i3(dims), _dp(img), _dp(out))
    return out


def prolong(nodes_c, ext_c, uc, nodes_f, ext_f):
    uc = _f64(uc)
    uf = np.empty((3, nodes_f[2], nodes_f[1], nodes_f[0]))
    lib().orc_prolong(_i3(nodes_c), _d3(ext_c), _dp(uc), _i3(nodes_f), _d3(ext_f), _dp(uf))
    return uf


def two_loop(S, Y, g, gamma):
    """H g for the L-BFGS matrix of pairs S[j], Y[j] (oldest first) with H0 = gamma I."""
    S, Y, g = _f64(S), _f64(Y), _f64(g)
    r = np.empty_like(g)
    lib().orc_two_loop(g.size, S.shape[0], _dp(S), _dp(Y), _dp(g), float(gamma), _dp(r))
    return r


def make_config(levels=1, tau=0.01, rho=None, alpha=10.0, mem=5, max_iter=50, c1=1e-4,
                max_backtracks=20, tol_grad_rel=1e-5, tol_j_rel=1e-7, tol_j_count=3,
                fixed_iters=False, start_level=-1, node_dims=None):
    cfg = Config()
    cfg.tau = tau
    cfg.rho = tau if rho is None else rho
    cfg.alpha = alpha
    cfg.c1 = c1
    cfg.tol_grad_rel = tol_grad_rel
    cfg.tol_j_rel = tol_j_rel
    cfg.tol_j_count = tol_j_count
    cfg.levels = levels
    cfg.mem = mem
    cfg.max_backtracks = max_backtracks
    cfg.fixed_iters = int(bool(fixed_iters))
    cfg.start_level = start_level
    its = max_iter if hasattr(max_iter, "__len__") else [max_iter] * MAX_LEVELS
    for lv in range(MAX_LEVELS):
        cfg.max_iter[lv] = int(its[lv]) if lv < len(its) else int(its[-1])
        for d in range(3):
            cfg.node_dims[lv][d] = 0 if node_dims is None else int(node_dims[lv][d])
    return cfg


def level_dims(dims, cfg, level):
    m, mn = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    lib().orc_level_dims(_i3(dims), ctypes.byref(cfg), int(level), m, mn)
    return tuple(m), tuple(mn)


def lbfgs_level(dims, spacing, R, T, nodes, cfg, max_iter, u0):
    R, T = _f64(R), _f64(T)
    u = _f64(u0).copy()
    it, ev, J = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().orc_lbfgs_level(_i3(dims), _d3(spacing), _dp(R), _dp(T), _i3(nodes), ctypes.byref(cfg),
                               int(max_iter), _dp(u), ctypes.byref(it), ctypes.byref(ev), ctypes.byref(J))
    return u, dict(iters=it.value, evals=ev.value, J=J.value, status=st)


def lbfgs(fun, x0, Hmin, cfg, max_iter):
    """The oracle's L-BFGS driver on any objective: fun(x) -> (J, g) for a
    float64 vector x.  Returns (x, dict(iters, evals, J, status)).  The level
    driver runs the same code with the objective of Eq. 1."""
    x = _f64(np.ravel(x0)).copy()
    n = x.size
    err = []

    def cb(_ctx, up, gp):
        try:
            xv = np.ctypeslib.as_array(up, shape=(n,)).copy()
            J, g = fun(xv)
            np.ctypeslib.as_array(gp, shape=(n,))[:] = np.asarray(g, dtype=np.float64).ravel()
            return float(J)
        except Exception as e:  # noqa: BLE001 - reported after the C call returns
            err.append(e)
            np.ctypeslib.as_array(gp, shape=(n,))[:] = 0.0
            return float("nan")

    cfun = EVAL_FN(cb)
    it, ev, J = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().orc_lbfgs(n, cfun, None, float(Hmin), ctypes.byref(cfg), int(max_iter), _dp(x), ctypes.byref(it),
                         ctypes.byref(ev), ctypes.byref(J))
    if err:
        raise err[0]
    return x, dict(iters=it.value, evals=ev.value, J=J.value, status=st)


def register(dims, spacing, R, T, cfg, u_init=None):
    """Multilevel registration; returns (u on the finest node grid, stats dict)."""
    R, T = _f64(R), _f64(T)
    _, mn0 = level_dims(dims, cfg, 0)
    u = np.empty((3, mn0[2], mn0[1], mn0[0]))
    st = Stats()
    ui = None if u_init is None else _dp(_f64(u_init))
    status = lib().orc_register(_i3(dims), _d3(spacing), _dp(R), _dp(T), ctypes.byref(cfg), ui, _dp(u),
                                ctypes.byref(st))
    L = cfg.levels
    stats = dict(status=status, iters=list(st.iters)[:L], evals=list(st.evals)[:L],
                 level_status=list(st.status)[:L], J=list(st.J)[:L])
    return u, stats
