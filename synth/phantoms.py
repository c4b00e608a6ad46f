"""Seeded synthetic image pairs shaped like the paper's workloads.

The paper measures on private follow-up CT scans and on the DIR-Lab 4D-CT
set (Sec. 3.1-3.2); neither is available, so these generators stand in for
them with the same shapes, spacings, intensity ranges and deformation sizes.

Every phantom is an analytic function f(x) of the physical position x (mm).
The reference image is R(x) = f(x) and the template is T(x) = f(x + d(x)) for
a known smooth displacement d, so the template is sampled exactly at the warped
positions and no image interpolation is involved.  Noise is added afterwards.
Images are returned as float32 arrays of shape (m_z, m_y, m_x) (x fastest),
voxel centres at x_d = (i_d + 1/2) h_d.

This module is shared by the tests, the benchmark and the examples.  It holds
none of the registration method's arithmetic.
"""
import numpy as np

from .configs import CONFIGS, seed_for, batch_sizes

HU_AIR = -1000.0
HU_SCALE = 1700.0


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def voxel_centres(dims, spacing, z0=0, z1=None):
    """Physical voxel-centre coordinates (X, Y, Z), each of shape (z1-z0, m_y, m_x)."""
    mx, my, mz = dims
    z1 = mz if z1 is None else z1
    hx, hy, hz = spacing
    z = (np.arange(z0, z1) + 0.5) * hz
    y = (np.arange(my) + 0.5) * hy
    x = (np.arange(mx) + 0.5) * hx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


# --------------------------------------------------------------------------
# analytic shapes
# --------------------------------------------------------------------------
class _Shape:
    """One smooth ellipsoid, ellipsoid shell or Gaussian blob."""

    def __init__(self, kind, centre, axes, value, thick=0.0, edge=1.0):
        self.kind = kind
        self.c = np.asarray(centre, float)
        self.a = np.asarray(axes, float)
        self.value = float(value)
        self.thick = float(thick)
        self.edge = float(edge)

    def reach(self):
        """Half-extent of the region where the shape is not negligible."""
        if self.kind == "blob":
            return 4.0 * self.a
        return self.a + self.thick + 4.0 * self.edge

    def weight(self, X, Y, Z):
        dx = (X - self.c[0]) / self.a[0]
        dy = (Y - self.c[1]) / self.a[1]
        dz = (Z - self.c[2]) / self.a[2]
        r2 = dx * dx + dy * dy + dz * dz
        if self.kind == "blob":
            return np.exp(-0.5 * r2)
        rho = np.sqrt(r2)
        amin = float(self.a.min())
        if self.kind == "ellipsoid":
            sd = (1.0 - rho) * amin
        else:  # shell
            sd = 0.5 * self.thick - np.abs(rho - 1.0) * amin
        return 0.5 * (1.0 + np.tanh(sd / self.edge))


class Phantom:
    """Layered analytic phantom: a background value, then shapes in order.

    Ellipsoids and shells replace the value below them (smoothly, with an edge
    width of about one voxel); blobs add to it.
    """

    def __init__(self, background, shapes, clip=None):
        self.background = float(background)
        self.shapes = list(shapes)
        self.clip = clip

    def __call__(self, X, Y, Z, margin=0.0):
        out = np.full(X.shape, self.background, dtype=np.float64)
        for s in self.shapes:
            lo = s.c - s.reach() - margin
            hi = s.c + s.reach() + margin
            sel = ((X >= lo[0]) & (X <= hi[0]) & (Y >= lo[1]) & (Y <= hi[1])
                   & (Z >= lo[2]) & (Z <= hi[2]))
            if not sel.any():
                continue
            w = s.weight(X[sel], Y[sel], Z[sel])
            if s.kind == "blob":
                out[sel] += s.value * w
            else:
                out[sel] = out[sel] * (1.0 - w) + s.value * w
        if self.clip is not None:
            np.clip(out, self.clip[0], self.clip[1], out=out)
        return out


# --------------------------------------------------------------------------
# displacement fields d(x) (mm); the template is T(x) = f(x + d(x))
# --------------------------------------------------------------------------
class ModeField:
    """Sum of sinusoidal modes A_j e_j sin(2 pi k_j . x / L + phi_j) plus an
    optional smooth breathing-like part, scaled to a prescribed maximum |d|."""

    def __init__(self, rng, extent, n_modes, max_k, breathing=None, mode_share=1.0):
        self.L = np.asarray(extent, float)
        self.k = rng.integers(-max_k, max_k + 1, size=(n_modes, 3)).astype(float)
        self.k[np.all(self.k == 0, axis=1), 0] = 1.0
        e = rng.normal(size=(n_modes, 3))
        self.e = e / np.linalg.norm(e, axis=1, keepdims=True)
        self.amp = rng.uniform(0.5, 1.0, size=n_modes)
        self.phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
        self.breathing = breathing
        self.mode_share = float(mode_share)
        self.scale = 1.0

    def __call__(self, X, Y, Z):
        d = np.zeros((3,) + X.shape)
        for k, e, a, ph in zip(self.k, self.e, self.amp, self.phase):
            arg = 2.0 * np.pi * (k[0] * X / self.L[0] + k[1] * Y / self.L[1]
                                 + k[2] * Z / self.L[2]) + ph
            s = a * np.sin(arg) * self.mode_share
            d[0] += e[0] * s
            d[1] += e[1] * s
            d[2] += e[2] * s
        if self.breathing is not None:
            d += self.breathing(X, Y, Z)
        return d * self.scale

    def normalise(self, dims, spacing, target_max):
        """Rescale so that max_x |d(x)| over the voxel centres equals target_max."""
        self.scale = 1.0
        mx = 0.0
        for z0 in range(0, dims[2], 16):
            X, Y, Z = voxel_centres(dims, spacing, z0, min(dims[2], z0 + 16))
            d = self(X, Y, Z)
            mx = max(mx, float(np.sqrt((d * d).sum(axis=0)).max()))
        self.scale = target_max / mx
        return self


class Breathing:
    """Craniocaudal (z) motion peaking at the diaphragm level with a smaller
    radial in-plane expansion; z grows toward the head."""

    def __init__(self, extent, cc=1.0, lateral=0.25, z_dia=0.40, z_apex=0.85, decay_apex=True):
        self.L = np.asarray(extent, float)
        self.cc, self.lat = cc, lateral
        self.z_dia, self.z_apex = z_dia, z_apex
        self.decay_apex = decay_apex

    def __call__(self, X, Y, Z):
        L = self.L
        xn = (X - 0.5 * L[0]) / (0.30 * L[0])
        yn = (Y - 0.5 * L[1]) / (0.30 * L[1])
        zn = Z / L[2]
        plane = np.exp(-0.5 * (xn * xn + yn * yn))
        if self.decay_apex:
            # full motion at and below the diaphragm, smooth decay to 0 at the apex
            t = np.clip((zn - self.z_dia) / (self.z_apex - self.z_dia), 0.0, 1.0)
            prof = 0.5 * (1.0 + np.cos(np.pi * t))
            prof *= np.exp(-0.5 * (np.minimum(zn - self.z_dia, 0.0) / 0.3) ** 2)
        else:
            prof = np.exp(-0.5 * ((zn - self.z_dia) / 0.25) ** 2)
        d = np.zeros((3,) + X.shape)
        d[2] = -self.cc * plane * prof
        d[0] = self.lat * xn * plane * prof
        d[1] = self.lat * yn * plane * prof
        return d


# --------------------------------------------------------------------------
# phantom builders
# --------------------------------------------------------------------------
def _blob_phantom(rng, dims, spacing):
    L = np.asarray(dims, float) * np.asarray(spacing, float)
    h = float(min(spacing))
    shapes = [_Shape("shell", 0.5 * L, [0.36 * L[0], 0.30 * L[1], 0.33 * L[2]], 0.8,
                     thick=3.0 * h, edge=0.7 * h)]
    for _ in range(20):
        c = rng.uniform(0.2, 0.8, size=3) * L
        sig = rng.uniform(2.0, 6.0) * h
        shapes.append(_Shape("blob", c, [sig, sig, sig], rng.uniform(0.2, 1.0)))
    return Phantom(0.0, shapes, clip=(0.0, 1.0))


def _ct_phantom(rng, dims, spacing, organs):
    """HU phantom: air, body, two lungs, heart, bone-like shells, organ ellipsoids."""
    L = np.asarray(dims, float) * np.asarray(spacing, float)
    h = float(min(spacing))
    e = 0.7 * h
    f = lambda *v: np.asarray(v, float) * L  # noqa: E731  (fractions of the extent)
    shapes = [
        _Shape("ellipsoid", f(0.5, 0.5, 0.5), f(0.42, 0.31, 0.47), -50.0, edge=e),
        _Shape("ellipsoid", f(0.33, 0.47, 0.62), f(0.12, 0.17, 0.22), -850.0, edge=e),
        _Shape("ellipsoid", f(0.67, 0.47, 0.62), f(0.12, 0.17, 0.22), -850.0, edge=e),
        _Shape("ellipsoid", f(0.53, 0.40, 0.52), f(0.09, 0.08, 0.08), 40.0, edge=e),
        _Shape("shell", f(0.5, 0.5, 0.62), f(0.37, 0.26, 0.28), 700.0, thick=0.012 * L.min(), edge=e),
        _Shape("shell", f(0.5, 0.74, 0.5), f(0.045, 0.045, 0.45), 700.0, thick=0.015 * L.min(), edge=e),
        _Shape("shell", f(0.5, 0.56, 0.12), f(0.26, 0.16, 0.07), 700.0, thick=0.015 * L.min(), edge=e),
    ]
    for _ in range(organs):
        c = f(rng.uniform(0.25, 0.75), rng.uniform(0.3, 0.7), rng.uniform(0.12, 0.42))
        ax = rng.uniform(5.0, 40.0, size=3)
        shapes.append(_Shape("ellipsoid", c, ax, 50.0 + rng.uniform(-60.0, 60.0), edge=e))
    return Phantom(HU_AIR, shapes)


def _lung_phantom(rng, dims, spacing):
    """Thorax HU phantom for the 4D-CT-shaped pair; lungs span the upper 60 %."""
    L = np.asarray(dims, float) * np.asarray(spacing, float)
    h = float(min(spacing))
    e = 0.7 * h
    f = lambda *v: np.asarray(v, float) * L  # noqa: E731
    lungs = [
        _Shape("ellipsoid", f(0.32, 0.48, 0.62), f(0.14, 0.19, 0.30), -850.0, edge=e),
        _Shape("ellipsoid", f(0.68, 0.48, 0.62), f(0.14, 0.19, 0.30), -850.0, edge=e),
    ]
    shapes = [
        _Shape("ellipsoid", f(0.5, 0.5, 0.5), f(0.44, 0.33, 0.60), -50.0, edge=e),
        *lungs,
        _Shape("ellipsoid", f(0.55, 0.42, 0.45), f(0.10, 0.09, 0.12), 40.0, edge=e),
        _Shape("shell", f(0.5, 0.5, 0.6), f(0.40, 0.29, 0.45), 700.0, thick=0.012 * L.min(), edge=e),
        _Shape("shell", f(0.5, 0.76, 0.5), f(0.045, 0.045, 0.6), 700.0, thick=0.015 * L.min(), edge=e),
    ]
    # vessel-like blobs inside the lungs give the NGF term texture to work with
    for _ in range(60):
        lung = lungs[int(rng.integers(0, 2))]
        dirn = rng.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        c = lung.c + dirn * lung.a * rng.uniform(0.0, 0.8)
        sig = rng.uniform(1.5, 4.0)
        shapes.append(_Shape("blob", c, [sig, sig, sig], rng.uniform(150.0, 500.0)))
    return Phantom(HU_AIR, shapes), lungs


# --------------------------------------------------------------------------
# sampling
# --------------------------------------------------------------------------
def _sample(phantom, dims, spacing, field=None, margin=0.0, slab=16):
    mx, my, mz = dims
    out = np.empty((mz, my, mx), dtype=np.float64)
    for z0 in range(0, mz, slab):
        z1 = min(mz, z0 + slab)
        X, Y, Z = voxel_centres(dims, spacing, z0, z1)
        if field is not None:
            d = field(X, Y, Z)
            X, Y, Z = X + d[0], Y + d[1], Z + d[2]
        out[z0:z1] = phantom(X, Y, Z, margin=margin)
    return out


def _hu_to_unit(hu):
    return np.clip((hu - HU_AIR) / HU_SCALE, 0.0, 1.0)


def make_pair(config_id, pair=0, dims=None):
    """Synthetic (R, T) pair of one workload.

    Returns a dict with float32 images ``R`` and ``T`` of shape (m_z, m_y, m_x),
    ``dims`` = (m_x, m_y, m_z), ``spacing`` (mm), the displacement ``field``
    d(x) used to make T (callable on physical coordinates), and for the
    4D-CT-shaped workload the landmark pairs ``lm_R`` and ``lm_T`` (mm).
    """
    cfg = CONFIGS[config_id]
    rng = _rng(seed_for(config_id, pair))
    dims = tuple(dims if dims is not None else cfg["dims"])
    spacing = tuple(cfg["spacing"])
    L = np.asarray(dims, float) * np.asarray(spacing, float)
    out = dict(dims=dims, spacing=spacing, config=config_id, pair=pair)
    kind = cfg["kind"]
    if kind == "blobs":
        ph = _blob_phantom(rng, dims, spacing)
        field = ModeField(rng, L, 8, 3).normalise(dims, spacing, cfg["max_disp_vox"] * min(spacing))
        margin = cfg["max_disp_vox"] * min(spacing)
        R = _sample(ph, dims, spacing)
        T = _sample(ph, dims, spacing, field, margin) + rng.normal(0.0, 0.01, size=(dims[2], dims[1], dims[0]))
        R, T = np.clip(R, 0, 1), np.clip(T, 0, 1)
    elif kind == "ct" and cfg.get("slab_noise"):
        ph, field = _ct_model(rng, dims, spacing, cfg)
        R, T = _ct_slab_pair(ph, field, dims, spacing, cfg, seed_for(config_id, pair), 0, dims[2])
    elif kind == "ct":
        ph, field = _ct_model(rng, dims, spacing, cfg)
        margin = cfg["max_disp_mm"]
        noise = lambda: rng.normal(0.0, 20.0, size=(dims[2], dims[1], dims[0]))  # noqa: E731
        R = _hu_to_unit(_sample(ph, dims, spacing) + noise())
        T = _hu_to_unit(_sample(ph, dims, spacing, field, margin) + noise())
    elif kind == "lung":
        ph, lungs = _lung_phantom(rng, dims, spacing)
        br = Breathing(L, cc=cfg["max_cc_mm"], lateral=cfg["max_lat_mm"], z_dia=0.32, z_apex=0.92)
        field = ModeField(rng, L, 1, 1, breathing=br, mode_share=0.0)
        margin = cfg["max_cc_mm"] + cfg["max_lat_mm"]
        noise = lambda: rng.normal(0.0, 20.0, size=(dims[2], dims[1], dims[0]))  # noqa: E731
        # int16 HU volumes, as a scanner writes them, then converted to [0, 1] FP32
        R16 = np.clip(np.rint(_sample(ph, dims, spacing) + noise()), -1024, 3071).astype(np.int16)
        T16 = np.clip(np.rint(_sample(ph, dims, spacing, field, margin) + noise()), -1024, 3071).astype(np.int16)
        out["R_hu"], out["T_hu"] = R16, T16
        R = _hu_to_unit(R16.astype(np.float64))
        T = _hu_to_unit(T16.astype(np.float64))
        lm_T, lm_R = _landmarks(rng, lungs, field, L, cfg["landmarks"])
        out["lm_R"], out["lm_T"] = lm_R, lm_T
    else:
        raise ValueError(kind)
    out["R"] = np.ascontiguousarray(R, dtype=np.float32)
    out["T"] = np.ascontiguousarray(T, dtype=np.float32)
    out["field"] = field
    return out


def _ct_model(rng, dims, spacing, cfg):
    """CT phantom and its breathing-like field (the draws every CT workload makes first)."""
    L = np.asarray(dims, float) * np.asarray(spacing, float)
    ph = _ct_phantom(rng, dims, spacing, cfg["organs"])
    field = ModeField(rng, L, 4, 2, breathing=Breathing(L, decay_apex=False), mode_share=0.2)
    field.normalise(dims, spacing, cfg["max_disp_mm"])
    return ph, field


def _ct_slab_pair(ph, field, dims, spacing, cfg, seed, z0, z1):
    """Planes z0 .. z1-1 of R and T of a slab-noise CT workload: noise of slab
    s = z // slab from its own PCG64 stream (seed * 4096 + s), so any split of
    the planes gives the same volume."""
    slab = int(cfg["slab_noise"])
    mx, my, _ = dims
    R = np.empty((z1 - z0, my, mx), dtype=np.float32)
    T = np.empty((z1 - z0, my, mx), dtype=np.float32)
    for s0 in range((z0 // slab) * slab, z1, slab):
        a, b = max(s0, z0), min(s0 + slab, z1)
        nrng = _rng(int(seed) * 4096 + s0 // slab)
        nR = nrng.normal(0.0, 20.0, size=(slab, my, mx))[a - s0:b - s0]
        nT = nrng.normal(0.0, 20.0, size=(slab, my, mx))[a - s0:b - s0]
        X, Y, Z = voxel_centres(dims, spacing, a, b)
        R[a - z0:b - z0] = _hu_to_unit(ph(X, Y, Z) + nR)
        d = field(X, Y, Z)
        T[a - z0:b - z0] = _hu_to_unit(ph(X + d[0], Y + d[1], Z + d[2], margin=cfg["max_disp_mm"]) + nT)
    return R, T


def _slab_job(job):
    config_id, pair, dims, z0, z1 = job
    cfg = CONFIGS[config_id]
    rng = _rng(seed_for(config_id, pair))
    spacing = tuple(cfg["spacing"])
    ph, field = _ct_model(rng, dims, spacing, cfg)
    return z0, _ct_slab_pair(ph, field, dims, spacing, cfg, seed_for(config_id, pair), z0, z1)


def make_pair_parallel(config_id, pair=0, dims=None, procs=None):
    """make_pair of a slab-noise workload, its planes generated by a spawn pool
    (the same arrays and field as make_pair)."""
    import multiprocessing as mp
    import os
    cfg = CONFIGS[config_id]
    dims = tuple(dims if dims is not None else cfg["dims"])
    slab = int(cfg["slab_noise"])
    jobs = [(config_id, pair, dims, z0, min(dims[2], z0 + slab)) for z0 in range(0, dims[2], slab)]
    procs = procs or min(len(jobs), os.cpu_count() or 1, 16)
    R = np.empty((dims[2], dims[1], dims[0]), dtype=np.float32)
    T = np.empty_like(R)
    with mp.get_context("spawn").Pool(procs) as pool:
        for z0, (r, t) in pool.imap_unordered(_slab_job, jobs):
            R[z0:z0 + r.shape[0]] = r
            T[z0:z0 + t.shape[0]] = t
    rng = _rng(seed_for(config_id, pair))
    ph, field = _ct_model(rng, dims, tuple(cfg["spacing"]), cfg)
    return dict(dims=dims, spacing=tuple(cfg["spacing"]), config=config_id, pair=pair, R=R, T=T, field=field)


def _landmarks(rng, lungs, field, extent, n):
    """Points p_T pushed through the known field: p_R = p_T + d(p_T).

    Because T(p_T) = f(p_T + d(p_T)) = R(p_R), the exact correspondence of the
    reference point p_R is p_T.  Points are kept only if p_R lies inside a lung.
    """
    keep_T, keep_R = [], []
    while len(keep_T) < n:
        p = rng.uniform(0.05, 0.95, size=(4 * n, 3)) * extent
        d = field(p[:, 0], p[:, 1], p[:, 2])
        q = p + d.T
        inside = np.zeros(len(p), bool)
        for lung in lungs:
            r = np.sqrt((((q - lung.c) / lung.a) ** 2).sum(axis=1))
            inside |= r < 0.9
        keep_T.extend(p[inside])
        keep_R.extend(q[inside])
    return np.asarray(keep_T[:n]), np.asarray(keep_R[:n])


def true_inverse_displacement(field, points, iters=50):
    """Displacement u(x) = y(x) - x of the exact correspondence y with
    y + d(y) = x (fixed-point iteration); points has shape (N, 3) in mm."""
    y = np.array(points, dtype=np.float64, copy=True)
    for _ in range(iters):
        d = field(y[:, 0], y[:, 1], y[:, 2])
        y = points - d.T
    return y - points


# --------------------------------------------------------------------------
# generic random inputs for unit and parity tests
# --------------------------------------------------------------------------
def random_image(dims, seed, n_blobs=12, smooth=True, noise=0.02):
    """Random image in [0, 1]: Gaussian blobs plus N(0, noise) (smooth) or uniform noise."""
    rng = _rng(seed)
    mx, my, mz = dims
    if not smooth:
        return rng.uniform(0.0, 1.0, size=(mz, my, mx)).astype(np.float32)
    L = np.asarray(dims, float)
    shapes = []
    for _ in range(n_blobs):
        c = rng.uniform(0.0, 1.0, size=3) * L
        sig = rng.uniform(0.08, 0.25) * L.min() + 0.8
        shapes.append(_Shape("blob", c, [sig, sig, sig], rng.uniform(-1.0, 1.0)))
    img = _sample(Phantom(0.5, shapes), dims, (1.0, 1.0, 1.0))
    img += noise * rng.normal(size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def random_field(node_dims, seed, amp):
    """Smooth random displacement on a node grid, shape (3, n_z, n_y, n_x), max |u_c| ~ amp."""
    rng = _rng(seed)
    nx, ny, nz = node_dims
    z, y, x = np.meshgrid(np.linspace(0, 1, nz), np.linspace(0, 1, ny), np.linspace(0, 1, nx), indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    for c in range(3):
        for _ in range(4):
            k = rng.uniform(0.5, 2.5, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            u[c] += np.sin(np.pi * k[0] * x + ph[0]) * np.sin(np.pi * k[1] * y + ph[1]) * np.sin(np.pi * k[2] * z + ph[2])
        u[c] *= amp / max(1e-12, np.abs(u[c]).max())
    return u.astype(np.float32)


def random_vector(n, seed):
    """Standard normal float64 vector of length n."""
    return _rng(seed).normal(size=n)


__all__ = ["make_pair", "random_image", "random_field", "random_vector", "voxel_centres",
           "true_inverse_displacement", "batch_sizes", "CONFIGS", "seed_for"]
