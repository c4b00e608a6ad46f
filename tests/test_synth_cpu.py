"""Input generators: seeded and reproducible pairs, the stated warp amplitude,
exact landmark correspondences of the 4D-CT-shaped pair, the inverse of a
known field, the uneven batch's size set, and the slab-parallel generation of
the full-resolution CT workload (any split of the planes draws the same
per-slab noise)."""
import numpy as np

from synth import make_pair, make_pair_parallel


def test_slab_parallel_generation_matches_serial():
    dims = (40, 36, 70)   # 70 planes: two full 32-plane slabs and a partial one
    a = make_pair(5, pair=1, dims=dims)
    b = make_pair_parallel(5, pair=1, dims=dims, procs=2)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["T"], b["T"])
    assert a["R"].shape == (70, 36, 40) and a["R"].dtype == np.float32
    assert 0.0 <= a["R"].min() and a["R"].max() <= 1.0


def test_pairs_are_seeded_and_reproducible():
    a, b = make_pair(0), make_pair(0)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["T"], b["T"])
    c = make_pair(0, pair=1)
    assert not np.array_equal(a["R"], c["R"])
    assert a["R"].shape == (64, 64, 64) and a["R"].dtype == np.float32
    assert 0.0 <= min(a["R"].min(), a["T"].min()) and max(a["R"].max(), a["T"].max()) <= 1.0


def test_64cube_warp_is_scaled_to_two_voxels():
    from synth import voxel_centres
    p = make_pair(0)
    X, Y, Z = voxel_centres(p["dims"], p["spacing"])
    d = p["field"](X, Y, Z)
    assert abs(np.sqrt((d * d).sum(axis=0)).max() - 2.0) < 1e-9


def test_4dct_landmarks_follow_the_known_field_exactly():
    """p_R = p_T + d(p_T), so T(p_T) = R(p_R) and the true correspondence of p_R is p_T."""
    p = make_pair(3, dims=(64, 64, 28))
    lm_R, lm_T = p["lm_R"], p["lm_T"]
    assert lm_R.shape == lm_T.shape == (300, 3)
    d = p["field"](lm_T[:, 0], lm_T[:, 1], lm_T[:, 2])
    np.testing.assert_allclose(lm_R - lm_T, d.T, rtol=0, atol=1e-12)
    extent = np.asarray(p["dims"]) * np.asarray(p["spacing"])
    assert (lm_T > 0).all() and (lm_T < extent).all() and (lm_R > 0).all() and (lm_R < extent).all()
    assert p["R_hu"].dtype == np.int16 and p["R_hu"].shape == (28, 64, 64)


def test_true_inverse_displacement_inverts_the_field():
    from synth import true_inverse_displacement
    p = make_pair(1, dims=(32, 32, 32))
    pts = np.random.default_rng(0).uniform(5.0, 40.0, size=(200, 3))
    u = true_inverse_displacement(p["field"], pts)
    y = pts + u
    d = p["field"](y[:, 0], y[:, 1], y[:, 2])
    np.testing.assert_allclose(y + d.T, pts, rtol=0, atol=1e-9)


def test_uneven_batch_sizes_come_from_the_size_set():
    from synth import CONFIGS, batch_sizes
    sizes = batch_sizes()
    allowed = set(CONFIGS[4]["size_set"])
    assert len(sizes) == 64 and set(sizes) <= allowed and len(set(sizes)) >= 4
    assert sizes == batch_sizes()
