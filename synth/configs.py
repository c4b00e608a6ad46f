"""Workload descriptions for the synthetic registration pairs.

Each entry fixes the image size, spacing and the solver parameters of one
workload.  The images themselves come from :mod:`synth.phantoms`.  Nothing in
this module computes any part of the registration method.

Solver parameters follow the paper's model (Budelmann et al., "Fully-deformable
3D image registration in two seconds", Sec. 2.1, Eq. 1-2): NGF edge
parameters tau = rho = eta, curvature weight alpha, L-BFGS memory, Armijo c1,
and an iteration cap per pyramid level.
"""

SEED_BASE = 181206765


def seed_for(config_id, pair=0):
    """Seed of one pair: SEED_BASE + 1000 * config + pair (numpy PCG64)."""
    return SEED_BASE + 1000 * int(config_id) + int(pair)


CONFIGS = {
    # single pair, single level, 64^3 at unit spacing, nodes 33^3
    0: dict(name="c0_64cube_1level", dims=(64, 64, 64), spacing=(1.0, 1.0, 1.0),
            levels=1, eta=0.01, alpha=10.0, mem=5, max_iter=50, c1=1e-4,
            kind="blobs", max_disp_vox=2.0),
    # CT-like 128^3 at 1.5 mm, 3 levels (32^3/64^3/128^3), nodes 17^3/33^3/65^3
    1: dict(name="c1_ct128_3level", dims=(128, 128, 128), spacing=(1.5, 1.5, 1.5),
            levels=3, eta=0.1, alpha=50.0, mem=5, max_iter=100, c1=1e-4,
            kind="ct", max_disp_mm=8.0, organs=0),
    # CT-like 256^3 at 1 mm plus 30 organ/tumour ellipsoids, 4 levels, nodes 129^3
    2: dict(name="c2_ct256_4level", dims=(256, 256, 256), spacing=(1.0, 1.0, 1.0),
            levels=4, eta=0.1, alpha=50.0, mem=5, max_iter=100, c1=1e-4,
            kind="ct", max_disp_mm=15.0, organs=30),
    # anisotropic thoracic 4D-CT shape, int16 HU, 4 levels, nodes 129x129x57
    3: dict(name="c3_lung256x256x112_4level", dims=(256, 256, 112),
            spacing=(0.97, 0.97, 2.5), levels=4, eta=0.1, alpha=50.0, mem=5,
            max_iter=100, c1=1e-4, kind="lung", max_cc_mm=20.0,
            max_lat_mm=5.0, landmarks=300),
    # full-resolution CT (the size the paper's GPU could not hold): 512^3 at 0.75 mm,
    # 5 levels, nodes 257^3; the noise is drawn per slab so slabs can be made apart
    5: dict(name="c5_ct512_fullres_5level", dims=(512, 512, 512), spacing=(0.75, 0.75, 0.75),
            levels=5, eta=0.1, alpha=50.0, mem=5, max_iter=100, c1=1e-4,
            kind="ct", max_disp_mm=15.0, organs=30, slab_noise=32),
    # batch of 64 uneven pairs at 1.5 mm, 3 levels, 60 iterations per level
    4: dict(name="c4_batch64_uneven", dims=None, spacing=(1.5, 1.5, 1.5),
            levels=3, eta=0.1, alpha=50.0, mem=5, max_iter=60, c1=1e-4,
            kind="ct", max_disp_mm=12.0, organs=10, pairs=64,
            size_set=((96, 96, 96), (128, 128, 128), (160, 160, 128),
                      (192, 192, 192), (224, 224, 160))),
}


def batch_sizes(n_pairs=64, seed=None):
    """Image dims of each pair of the uneven batch, drawn uniformly from the size set."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed_for(4, 10_000) if seed is None else seed))
    sizes = CONFIGS[4]["size_set"]
    return [tuple(sizes[int(k)]) for k in rng.integers(0, len(sizes), size=n_pairs)]
