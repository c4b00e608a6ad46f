"""Pins of the FP64 oracle against facts the mathematics fixes.

Each test compares the oracle with something other than itself: closed forms,
invariants, an independent library construction (numpy.interp, scipy's
map_coordinates, scipy.sparse Kronecker products, numpy reshape-means, the
dense BFGS update) or hand-derived tables.  The choice is such that a dropped
term, a wrong sign, a wrong index or a transposed operand anywhere in the
oracle fails at least one of them.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from synth import random_image, random_field, random_vector

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def node_coords(nodes, H):
    nx, ny, nz = nodes
    Z, Y, X = np.meshgrid(np.arange(nz) * H[2], np.arange(ny) * H[1], np.arange(nx) * H[0], indexing="ij")
    return X, Y, Z


def voxel_coords(dims, h):
    mx, my, mz = dims
    Z, Y, X = np.meshgrid((np.arange(mz) + 0.5) * h[2], (np.arange(my) + 0.5) * h[1],
                          (np.arange(mx) + 0.5) * h[0], indexing="ij")
    return X, Y, Z


CASES = [((16, 16, 16), (1.0, 1.0, 1.0), (9, 9, 9)),
         ((17, 12, 9), (0.9, 1.3, 2.5), (9, 7, 5)),      # non-integer ratios, anisotropic
         ((16, 8, 12), (1.0, 1.0, 1.0), (5, 5, 4))]      # ratio 4 and 2 and 4


# --------------------------------------------------------------------------
# grid conversion P and its adjoint (Eq. 1, Eq. 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims,h,nodes", CASES)
def test_P_reproduces_affine(orc, dims, h, nodes):
    H = orc.node_spacing(dims, h, nodes)
    Xn, Yn, Zn = node_coords(nodes, H)
    Xv, Yv, Zv = voxel_coords(dims, h)
    A = np.array([0.3, -1.7, 0.45])
    u = A[0] * Xn + A[1] * Yn + A[2] * Zn - 2.5
    ref = A[0] * Xv + A[1] * Yv + A[2] * Zv - 2.5
    np.testing.assert_allclose(orc.P(dims, h, nodes, u), ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.P(dims, h, nodes, np.ones_like(u)), 1.0, rtol=0, atol=1e-14)


def _P_dense_kron(dims, h, nodes):
    """Dense P built as a Kronecker product of 1D linear-interpolation matrices
    obtained from numpy.interp of unit vectors (independent of the oracle)."""
    mats = []
    for d in range(3):
        H = dims[d] * h[d] / (nodes[d] - 1)
        xn = np.arange(nodes[d]) * H
        xv = (np.arange(dims[d]) + 0.5) * h[d]
        mats.append(np.stack([np.interp(xv, xn, e) for e in np.eye(nodes[d])], axis=1))
    return np.kron(mats[2], np.kron(mats[1], mats[0]))


@pytest.mark.parametrize("dims,h,nodes", [((4, 4, 4), (1.0, 1.0, 1.0), (3, 3, 3)),
                                          ((5, 4, 6), (1.0, 2.0, 0.5), (3, 3, 4))])
def test_P_dense_brute_force(orc, dims, h, nodes):
    Pd = _P_dense_kron(dims, h, nodes)
    nn = int(np.prod(nodes))
    cols = np.stack([orc.P(dims, h, nodes, e.reshape(nodes[::-1])).ravel() for e in np.eye(nn)], axis=1)
    np.testing.assert_allclose(cols, Pd, rtol=0, atol=1e-14)
    # P^T is the transpose of the same matrix
    nv = int(np.prod(dims))
    rows = np.stack([orc.PT(dims, h, nodes, e.reshape(dims[::-1])).ravel() for e in np.eye(nv)], axis=0)
    np.testing.assert_allclose(rows, Pd, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dims,h,nodes", CASES)
def test_PT_adjoint_identity(orc, dims, h, nodes):
    x = random_vector(int(np.prod(nodes)), 11).reshape(nodes[::-1])
    z = random_vector(int(np.prod(dims)), 12).reshape(dims[::-1])
    lhs = float(np.vdot(orc.P(dims, h, nodes, x), z))
    rhs = float(np.vdot(x, orc.PT(dims, h, nodes, z)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_PT_of_ones_closed_form(orc):
    # ratio 2: each node collects weights 1/4,3/4,3/4,1/4 (sum 2) per dim, boundary nodes 3/4,1/4 (sum 1)
    dims, h, nodes = (16, 12, 8), (1.0, 1.0, 1.0), (9, 7, 5)
    out = orc.PT(dims, h, nodes, np.ones(dims[::-1]))
    s = [np.where((np.arange(n) == 0) | (np.arange(n) == n - 1), 1.0, 2.0) for n in nodes]
    ref = s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14)


def test_PT_tables_golden(orc):
    with open(os.path.join(GOLDEN, "pt_tables.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        m, mn, k, first = int(r[0]), int(r[1]), int(r[2]), int(r[3])
        w_ref = np.array([float(Fraction(w)) for w in r[4:]])
        f, w = orc.PT_table(m, 1.0, mn, k)
        assert f == first, r
        np.testing.assert_allclose(w, w_ref, rtol=0, atol=1e-14, err_msg=str(r))


# --------------------------------------------------------------------------
# template interpolation
# --------------------------------------------------------------------------
def test_interp_matches_scipy_zero_extension(orc):
    from scipy.ndimage import map_coordinates
    dims, h = (9, 7, 6), (1.2, 0.8, 2.0)
    T = random_image(dims, 5, smooth=False).astype(np.float64)
    rng = np.random.default_rng(3)
    L = np.array(dims) * np.array(h)
    pts = rng.uniform(-0.3, 1.3, size=(4000, 3)) * L        # includes points outside the box
    val, _ = orc.interp(dims, h, T, pts)
    idx = (pts / np.array(h) - 0.5)[:, ::-1].T                # (z, y, x) index coordinates
    ref = map_coordinates(T, idx, order=1, mode="grid-constant", cval=0.0)
    np.testing.assert_allclose(val, ref, rtol=0, atol=1e-12)


def test_interp_affine_and_nodes(orc):
    dims, h = (8, 6, 5), (1.0, 1.5, 2.0)
    Xv, Yv, Zv = voxel_coords(dims, h)
    A = np.array([0.7, -0.2, 1.1])
    T = A[0] * Xv + A[1] * Yv + A[2] * Zv + 0.3
    rng = np.random.default_rng(4)
    lo = 0.5 * np.array(h)
    hi = (np.array(dims) - 0.5) * np.array(h)
    pts = rng.uniform(lo, hi, size=(2000, 3))
    val, grad = orc.interp(dims, h, T, pts)
    np.testing.assert_allclose(val, pts @ A + 0.3, rtol=0, atol=1e-12)
    np.testing.assert_allclose(grad, np.broadcast_to(A, grad.shape), rtol=0, atol=1e-12)
    # at voxel centres the interpolant returns the voxel values
    centres = np.stack([Xv.ravel(), Yv.ravel(), Zv.ravel()], axis=1)
    val, _ = orc.interp(dims, h, T, centres)
    np.testing.assert_allclose(val, T.ravel(), rtol=0, atol=1e-12)
    # zero extension: at the box corner p = 0 the value is (1/2)^3 T_000
    val, _ = orc.interp(dims, h, T, np.zeros((1, 3)))
    assert abs(val[0] - 0.125 * T[0, 0, 0]) < 1e-14


def test_interp_gradient_is_derivative_of_value(orc):
    dims, h = (7, 8, 9), (1.0, 0.7, 1.3)
    T = random_image(dims, 8, smooth=False).astype(np.float64)
    rng = np.random.default_rng(9)
    pts = rng.uniform(0.0, 1.0, size=(500, 3)) * np.array(dims) * np.array(h)
    _, grad = orc.interp(dims, h, T, pts)
    eps = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = eps
        vp, _ = orc.interp(dims, h, T, pts + e)
        vm, _ = orc.interp(dims, h, T, pts - e)
        fd = (vp - vm) / (2 * eps)
        # skip the few points within eps of a cell face (the interpolant has a kink there)
        t = pts[:, d] / h[d] - 0.5
        ok = np.abs(t - np.rint(t)) > 1e-4
        np.testing.assert_allclose(grad[ok, d], fd[ok], rtol=0, atol=1e-7)


# --------------------------------------------------------------------------
# NGF (Eq. 2)
# --------------------------------------------------------------------------
def _interior_central_diff(img, h):
    b = [(img[1:-1, 1:-1, 2:] - img[1:-1, 1:-1, :-2]) / (2 * h[0]),
         (img[1:-1, 2:, 1:-1] - img[1:-1, :-2, 1:-1]) / (2 * h[1]),
         (img[2:, 1:-1, 1:-1] - img[:-2, 1:-1, 1:-1]) / (2 * h[2])]
    return np.stack(b)


def test_ngf_T_equals_R(orc):
    dims, h = (12, 10, 9), (1.0, 1.2, 0.8)
    R = random_image(dims, 21).astype(np.float64)
    nodes = (7, 6, 5)
    u = np.zeros((3,) + nodes[::-1])
    J, D, S, g = orc.objective(dims, h, R, R, nodes, u, 0.05, 0.05, 3.0)
    assert abs(D) < 1e-12 and abs(S) == 0.0
    assert np.abs(g).max() < 1e-12


def test_ngf_T_minus_R_closed_form(orc):
    dims, h, eta = (12, 10, 9), (1.0, 1.2, 0.8), 0.07
    R = random_image(dims, 22).astype(np.float64)
    D, _ = orc.ngf(dims, h, -R, R, eta, eta)
    b = _interior_central_diff(R, h)
    bb = (b * b).sum(axis=0)
    ref = 0.5 * np.prod(h) * np.sum(4 * eta**2 * bb / (bb + eta**2) ** 2)
    assert abs(D - ref) <= 1e-12 * abs(ref)


def test_ngf_linear_ramps_closed_form(orc):
    dims, h, tau, rho = (10, 9, 8), (1.0, 1.5, 0.5), 0.3, 0.2
    X, Y, Z = voxel_coords(dims, h)
    a = np.array([0.4, -0.1, 0.25])
    b = np.array([-0.2, 0.3, 0.15])
    T = a[0] * X + a[1] * Y + a[2] * Z
    R = b[0] * X + b[1] * Y + b[2] * Z
    D, v = orc.ngf(dims, h, T, R, tau, rho)
    na, nb = np.sqrt(a @ a + tau**2), np.sqrt(b @ b + rho**2)
    c = (a @ b + tau * rho) / (na * nb)
    n_int = (dims[0] - 2) * (dims[1] - 2) * (dims[2] - 2)
    assert abs(D - 0.5 * np.prod(h) * n_int * (1 - c * c)) < 1e-12 * n_int
    # v at interior voxels is the derivative of 1 - c^2 w.r.t. a (checked by FD on c)
    def psi(av):
        cc = (av @ b + tau * rho) / (np.sqrt(av @ av + tau**2) * nb)
        return 1 - cc * cc
    fd = np.array([(psi(a + e) - psi(a - e)) / 2e-6 for e in np.eye(3) * 1e-6])
    np.testing.assert_allclose(v[:, 4, 4, 4], fd, rtol=1e-7, atol=1e-10)
    assert np.all(v[:, 0] == 0) and np.all(v[:, :, :, -1] == 0)


def test_integer_voxel_shift_is_global_minimum(orc):
    # T is R shifted by s voxels; the constant displacement u = s h maps it back,
    # so J = 0 and grad J = 0.  Pins the sign of the deformation (x + yhat).
    dims, h = (20, 18, 16), (1.0, 1.5, 2.0)
    s = np.array([2, -1, 1])
    R = np.zeros(dims[::-1])
    R[4:-4, 4:-4, 4:-4] = random_image((dims[0] - 8, dims[1] - 8, dims[2] - 8), 31).astype(np.float64)
    T = np.roll(R, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))     # T_j = R_{j - s}
    nodes = (11, 10, 9)
    u = np.stack([np.full(nodes[::-1], s[d] * h[d]) for d in range(3)])
    J, D, S, g = orc.objective(dims, h, R, T, nodes, u, 0.02, 0.02, 5.0)
    assert abs(J) < 1e-12 and np.abs(g).max() < 1e-10
    # and the opposite sign is far from it
    J2, *_ = orc.objective(dims, h, R, T, nodes, -u, 0.02, 0.02, 5.0)
    assert J2 > 1.0


# --------------------------------------------------------------------------
# curvature regulariser
# --------------------------------------------------------------------------
def _laplacian_kron(nodes, H):
    """7-point Laplacian as scipy.sparse Kronecker sums, rows restricted to interior nodes."""
    import scipy.sparse as sp

    def d2(n, Hd):
        return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / Hd**2

    Ix, Iy, Iz = (sp.identity(n) for n in nodes)
    L = (sp.kron(Iz, sp.kron(Iy, d2(nodes[0], H[0]))) + sp.kron(Iz, sp.kron(d2(nodes[1], H[1]), Ix))
         + sp.kron(d2(nodes[2], H[2]), sp.kron(Iy, Ix)))
    mask = np.zeros(nodes[::-1], bool)
    mask[1:-1, 1:-1, 1:-1] = True
    return sp.csr_matrix(sp.diags(mask.ravel().astype(float)) @ L)


def test_curvature_affine_is_zero(orc):
    nodes, H = (7, 6, 5), (1.5, 2.0, 2.5)
    X, Y, Z = node_coords(nodes, H)
    u = np.stack([0.1 * X - 0.3 * Z + 1, 0.2 * Y + 0.05 * X, -0.4 * Z + 0.7 * Y - 3])
    S, g = orc.curvature(nodes, H, u)
    assert abs(S) < 1e-20 and np.abs(g).max() < 1e-12


def test_curvature_quadratic_and_sine_mode(orc):
    nodes, H = (9, 8, 7), (1.5, 2.0, 2.5)
    X, Y, Z = node_coords(nodes, H)
    n_int = (nodes[0] - 2) * (nodes[1] - 2) * (nodes[2] - 2)
    hy = np.prod(H)
    S, _ = orc.curvature(nodes, H, np.stack([X**2, Y**2, Z**2]))
    assert abs(S - 0.5 * hy * 3 * 4 * n_int) < 1e-9 * S
    # discrete eigenfunction of the interior stencil: sin(pi k j / (n-1)) per dim
    k = (2, 1, 3)
    jx, jy, jz = (np.arange(n) for n in nodes)
    mode = (np.sin(np.pi * k[2] * jz / (nodes[2] - 1))[:, None, None]
            * np.sin(np.pi * k[1] * jy / (nodes[1] - 1))[None, :, None]
            * np.sin(np.pi * k[0] * jx / (nodes[0] - 1))[None, None, :])
    lam = sum((2 * np.cos(np.pi * k[d] / (nodes[d] - 1)) - 2) / H[d] ** 2 for d in range(3))
    u = np.stack([mode, 0 * mode, 0 * mode])
    S, _ = orc.curvature(nodes, H, u)
    ref = 0.5 * hy * lam**2 * np.sum(mode[1:-1, 1:-1, 1:-1] ** 2)
    assert abs(S - ref) < 1e-10 * ref


def test_curvature_gradient_matches_sparse_construction(orc):
    nodes, H = (8, 7, 6), (1.0, 1.7, 2.2)
    L = _laplacian_kron(nodes, H)
    u = random_field(nodes, 41, 2.0).astype(np.float64)
    S, g = orc.curvature(nodes, H, u)
    hy = np.prod(H)
    S_ref = 0.0
    for c in range(3):
        w = L @ u[c].ravel()
        S_ref += 0.5 * hy * (w @ w)
        np.testing.assert_allclose(g[c].ravel(), hy * (L.T @ w), rtol=0, atol=1e-10 * np.abs(g).max())
    assert abs(S - S_ref) < 1e-12 * S_ref


# --------------------------------------------------------------------------
# whole objective: analytic gradient against central finite differences
# --------------------------------------------------------------------------
@pytest.mark.parametrize("aniso", [False, True])
def test_objective_gradient_finite_differences(orc, aniso):
    dims = (16, 16, 16)
    h = (1.3, 0.9, 1.6) if aniso else (1.0, 1.0, 1.0)
    nodes = (9, 9, 9)
    R = random_image(dims, 51).astype(np.float64)
    T = random_image(dims, 52).astype(np.float64)
    u = random_field(nodes, 53, 1.3).astype(np.float64)
    tau, rho, alpha = 0.08, 0.05, 0.7
    J, D, S, g = orc.objective(dims, h, R, T, nodes, u, tau, rho, alpha)
    eps = 1e-6
    fd = np.empty(u.size)
    uf = u.ravel()
    for q in range(u.size):
        old = uf[q]
        uf[q] = old + eps
        Jp = orc.objective(dims, h, R, T, nodes, u, tau, rho, alpha)[0]
        uf[q] = old - eps
        Jm = orc.objective(dims, h, R, T, nodes, u, tau, rho, alpha)[0]
        uf[q] = old
        fd[q] = (Jp - Jm) / (2 * eps)
    rel = np.linalg.norm(fd - g.ravel()) / np.linalg.norm(g)
    assert rel < 1e-6, rel


# --------------------------------------------------------------------------
# pyramid and prolongation
# --------------------------------------------------------------------------
def test_restrict_is_block_mean(orc):
    dims = (10, 8, 6)
    img = random_image(dims, 61, smooth=False).astype(np.float64)
    out = orc.restrict(dims, img)
    ref = img.reshape(3, 2, 4, 2, 5, 2).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-15)
    assert abs(out.mean() - img.mean()) < 1e-14
    np.testing.assert_allclose(orc.restrict(dims, np.full(dims[::-1], 0.37)), 0.37, atol=1e-15)


def test_restrict_odd_replicates_last_slab(orc):
    dims = (5, 2, 2)
    img = np.arange(20, dtype=np.float64).reshape(2, 2, 5)
    out = orc.restrict(dims, img)
    assert out.shape == (1, 1, 3)
    padded = np.concatenate([img, img[:, :, -1:]], axis=2)
    ref = padded.reshape(1, 2, 1, 2, 3, 2).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(out, ref, atol=1e-14)


def test_prolong_affine_and_nesting(orc):
    nc, nf = (9, 7, 5), (17, 13, 9)
    ext = (32.0, 24.0, 16.0)
    Hc = tuple(ext[d] / (nc[d] - 1) for d in range(3))
    Hf = tuple(ext[d] / (nf[d] - 1) for d in range(3))
    Xc, Yc, Zc = node_coords(nc, Hc)
    Xf, Yf, Zf = node_coords(nf, Hf)
    aff = lambda X, Y, Z: np.stack([0.2 * X - Z, 0.1 * Y + 3, X + Y + Z])  # noqa: E731
    uf = orc.prolong(nc, ext, aff(Xc, Yc, Zc), nf, ext)
    np.testing.assert_allclose(uf, aff(Xf, Yf, Zf), rtol=0, atol=1e-12)
    uc = random_field(nc, 71, 1.0).astype(np.float64)
    uf = orc.prolong(nc, ext, uc, nf, ext)
    np.testing.assert_array_equal(uf[:, ::2, ::2, ::2], uc)


# --------------------------------------------------------------------------
# L-BFGS
# --------------------------------------------------------------------------
def test_two_loop_equals_dense_bfgs_inverse(orc):
    n, m = 10, 4
    rng = np.random.default_rng(81)
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)       # SPD so that s'y > 0
    S = rng.normal(size=(m, n))
    Y = S @ A.T
    g = rng.normal(size=n)
    gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    Hm = gamma * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        Hm = V.T @ Hm @ V + rho * np.outer(s, s)
    np.testing.assert_allclose(orc.two_loop(S, Y, g, gamma), Hm @ g, rtol=1e-12, atol=1e-12)


def test_lbfgs_converges_to_quadratic_minimiser(orc):
    # R = T = 0 makes D identically 0 (c = 1, v = 0), leaving J = alpha S(u), a
    # convex quadratic with Hessian A = alpha hbar_y L^T M L.  Iterates stay in
    # u0 + range(A), so the limit is u0 minus its component in range(A).
    dims, h, nodes = (10, 10, 10), (1.0, 1.0, 1.0), (6, 6, 6)
    H = orc.node_spacing(dims, h, nodes)
    zero = np.zeros(dims[::-1])
    u0 = random_field(nodes, 91, 1.0).astype(np.float64)
    alpha = 2.0
    cfg = orc.make_config(levels=1, tau=0.1, alpha=alpha, mem=5, max_iter=400, tol_grad_rel=1e-11,
                          tol_j_rel=0.0, tol_j_count=1000)
    u, st = orc.lbfgs_level(dims, h, zero, zero, nodes, cfg, 400, u0)
    L = _laplacian_kron(nodes, H).toarray()
    A = alpha * np.prod(H) * L.T @ L
    Ap = np.linalg.pinv(A, rcond=1e-12)
    for c in range(3):
        ref = u0[c].ravel() - Ap @ (A @ u0[c].ravel())
        np.testing.assert_allclose(u[c].ravel(), ref, rtol=0, atol=1e-6)
    assert st["status"] == 0


def test_objective_on_cell_faces_takes_the_right_cell(orc):
    """At u = 0 every sample sits on a voxel centre, i.e. on a cell face of the
    interpolant; R5 takes the cell to its right there, so grad T is the forward
    difference (T_{i+1} - T_i) / h with T = 0 past the last voxel.  The objective's
    gradient must equal P^T (g grad T) assembled from that definition, also for
    spacings that are not dyadic fractions: with h = 2.4 mm, forming the
    coordinate through the physical position, (i + 1/2) h / h - 1/2, rounds below
    the integer for i = 15 and 28."""
    dims, h = (32, 9, 8), (2.4, 2.0, 3.0)
    nodes = orc.default_nodes(dims)
    rng = np.random.default_rng(7)
    R = rng.random((dims[2], dims[1], dims[0]))
    T = rng.random((dims[2], dims[1], dims[0]))
    tau = rho = 0.05
    u = np.zeros((3, nodes[2], nodes[1], nodes[0]))
    J, D, S, grad = orc.objective(dims, h, R, T, nodes, u, tau, rho, 1.0)
    D_ref, v = orc.ngf(dims, h, T, R, tau, rho)        # the deformed template is T itself
    g = orc.ngf_adjoint(dims, h, v)
    dT = []
    for ax, hd in zip((2, 1, 0), h):                     # axes of x, y, z in (z, y, x) arrays
        nxt = np.roll(T, -1, axis=ax)
        idx = [slice(None)] * 3
        idx[ax] = -1
        nxt[tuple(idx)] = 0.0                            # zero extension
        dT.append((nxt - T) / hd)
    ref = np.stack([orc.PT(dims, h, nodes, g * dT[c]) for c in range(3)])
    assert D == pytest.approx(D_ref, rel=1e-14) and S == 0.0
    np.testing.assert_allclose(grad, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.fixture
def compensated(orc):
    orc.set_compensated_sums(True)
    yield orc
    orc.set_compensated_sums(False)


def test_reduction_plain_and_compensated_definitions(orc, compensated):
    """Compensated sums are exact where the running sum loses a term to rounding;
    on many terms they match the correctly rounded sum (math.fsum, Shewchuk's
    exact summation) to one rounding."""
    import math
    a = np.array([1e16, 1.0, -1e16])
    assert compensated.reduce_sum(a) == 1.0
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.standard_normal(200_000) * 10.0 ** rng.integers(-8, 9, 200_000)
    exact = math.fsum(x)
    assert abs(compensated.reduce_sum(x) - exact) <= 2 * np.spacing(abs(exact))
    orc.set_compensated_sums(False)
    assert orc.reduce_sum(a) == 0.0                              # (1e16 + 1) rounds to 1e16
    assert orc.reduce_sum(x) == float(np.cumsum(x)[-1])          # the running sum in index order


def test_objective_reduction_order_is_far_below_the_tolerances(orc):
    """The FP64 objective with compensated reductions agrees with the plain
    index-order sums to 1e-12: the oracle's own rounding is negligible against
    the 1e-5 (J) and 1e-4 (grad) parity tolerances."""
    dims, h = (40, 36, 28), (1.0, 1.1, 0.9)
    R = random_image(dims, 61).astype(np.float64)
    T = random_image(dims, 62).astype(np.float64)
    nodes = (21, 19, 15)
    u = random_field(nodes, 63, 2.0).astype(np.float64)
    plain = orc.objective(dims, h, R, T, nodes, u, 0.05, 0.05, 5.0)
    orc.set_compensated_sums(True)
    try:
        comp = orc.objective(dims, h, R, T, nodes, u, 0.05, 0.05, 5.0)
    finally:
        orc.set_compensated_sums(False)
    for a, b in zip(plain[:3], comp[:3]):
        assert abs(a - b) <= 1e-12 * abs(b)
    assert np.array_equal(plain[3], comp[3])   # the gradient holds no global reduction


def test_failed_line_search_ends_the_level_with_the_warning(orc):
    """R9 on the convex quadratic J = alpha S (R = T = 0): along any descent
    direction J(u + t p) = J + t g'p + t^2 p'Ap / 2, so the Armijo test with c1
    within 1e-9 of 1 fails for every trial t >= 1/4.  The first search (the p0
    direction) uses its max_backtracks trials, the level ends with the warning
    status, no step is accepted and u stays u0."""
    dims, h, nodes = (10, 10, 10), (1.0, 1.0, 1.0), (6, 6, 6)
    zero = np.zeros(dims[::-1])
    u0 = random_field(nodes, 92, 1.0).astype(np.float64)
    for trials in (1, 3):
        cfg = orc.make_config(levels=1, tau=0.1, alpha=2.0, mem=5, max_iter=10, c1=1.0 - 1e-9,
                              max_backtracks=trials)
        u, st = orc.lbfgs_level(dims, h, zero, zero, nodes, cfg, 10, u0)
        assert st["status"] == 1 and st["iters"] == 0
        assert st["evals"] == 1 + trials        # the objective at u0, then one per trial
        assert np.array_equal(u, u0)
    # the same problem with the default c1 takes its steps
    cfg = orc.make_config(levels=1, tau=0.1, alpha=2.0, mem=5, max_iter=10)
    u, st = orc.lbfgs_level(dims, h, zero, zero, nodes, cfg, 10, u0)
    assert st["status"] == 0 and st["iters"] >= 1 and st["J"] < orc.objective(dims, h, zero, zero, nodes, u0, 0.1,
                                                                               0.1, 2.0)[0]


def test_multilevel_register_is_levels_joined_by_prolongation(orc):
    """Sec. 2.1's coarse-to-fine scheme: an affine start field has S = 0 and, with
    R = T = 0, a zero gradient, so no level iterates and the result is the same
    affine field on the finest nodes (prolongation reproduces affine fields;
    node spacings 4, 6, 8 mm and 2, 3, 4 mm keep every value exact).
    With images, the multilevel driver equals its pieces run by hand: L-BFGS on
    the 2x2x2-mean level, nodal prolongation onto the finer nodes of the same box,
    L-BFGS on the finest level."""
    dims, h = (20, 16, 12), (1.0, 1.5, 2.0)
    cfg = orc.make_config(levels=2, tau=0.05, alpha=3.0, mem=4, max_iter=[5, 7])
    (mc, nc), (_, nf) = orc.level_dims(dims, cfg, 1), orc.level_dims(dims, cfg, 0)
    ext = tuple(dims[d] * h[d] for d in range(3))
    Hc = tuple(ext[d] / (nc[d] - 1) for d in range(3))
    Hf = tuple(ext[d] / (nf[d] - 1) for d in range(3))
    # dyadic coefficients on integer node coordinates: every second difference is exactly 0
    aff = lambda X, Y, Z: np.stack([0.125 * X - 0.0625 * Z + 0.25, 0.0625 * Y, -0.03125 * X + 0.125 * Z])  # noqa: E731
    zero = np.zeros(dims[::-1])
    u, st = orc.register(dims, h, zero, zero, cfg, u_init=aff(*node_coords(nc, Hc)))
    assert st["status"] == 0 and st["iters"] == [0, 0]
    np.testing.assert_allclose(u, aff(*node_coords(nf, Hf)), rtol=0, atol=1e-12)

    R = random_image(dims, 101).astype(np.float64)
    T = np.roll(R, shift=(1, -1, 1), axis=(0, 1, 2))
    u0 = random_field(nc, 102, 0.5).astype(np.float64)
    u, st = orc.register(dims, h, R, T, cfg, u_init=u0)
    hc = tuple(2 * v for v in h)
    u1, s1 = orc.lbfgs_level(mc, hc, orc.restrict(dims, R), orc.restrict(dims, T), nc, cfg, 7, u0)
    uf, s0 = orc.lbfgs_level(dims, h, R, T, nf, cfg, 5, orc.prolong(nc, ext, u1, nf, ext))
    assert st["iters"] == [s0["iters"], s1["iters"]] and st["evals"] == [s0["evals"], s1["evals"]]
    assert s1["iters"] >= 1 and s0["iters"] >= 1
    np.testing.assert_array_equal(u, uf)


def test_oracle_result_does_not_depend_on_the_thread_count(orc):
    """OpenMP only splits independent per-voxel and per-node maps and every sum
    runs sequentially in index order, so one thread and all threads give the
    same bits."""
    import json
    import subprocess
    import sys
    code = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from synth import random_image, random_field
dims, h = (24, 20, 18), (1.0, 1.2, 0.9)
R, T = random_image(dims, 1).astype(np.float64), random_image(dims, 2).astype(np.float64)
nodes = oracle.default_nodes(dims)
J, D, S, g = oracle.objective(dims, h, R, T, nodes, random_field(nodes, 3, 0.8).astype(np.float64), 0.05, 0.05, 1.0)
import hashlib
print(json.dumps({"J": J.hex(), "D": D.hex(), "S": S.hex(), "g": hashlib.sha256(g.tobytes()).hexdigest(),
                  "threads": oracle.num_threads()}))
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        r = subprocess.run([sys.executable, "-c", code, root], capture_output=True, text=True, env=env,
                           timeout=300, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert outs[0]["threads"] == 1 and outs[1]["threads"] == 4
    for key in ("J", "D", "S", "g"):
        assert outs[0][key] == outs[1][key], key
