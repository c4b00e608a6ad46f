"""Landmark error on the 4D-CT-shaped pair (256 x 256 x 112, 0.97 x 0.97 x 2.5 mm).

The synthetic landmarks are exact correspondences (p_T pushed through the known
field gives p_R), so the mean landmark error after registration measures how
well the registration recovers the deformation; it is reported with the wall
time, the way the paper reports DIR-Lab results (Sec. 3.2).
"""
import time

import numpy as np
import pytest

from synth import CONFIGS, make_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _u_at(u, points, node_spacing):
    """Nodal trilinear value of u (3, n_z, n_y, n_x) at points (N, 3) in mm."""
    from scipy.ndimage import map_coordinates
    idx = (np.asarray(points) / np.asarray(node_spacing))[:, ::-1].T    # (z, y, x) node coordinates
    return np.stack([map_coordinates(u[c].astype(np.float64), idx, order=1, mode="nearest") for c in range(3)], 1)


@pytest.mark.slow
def test_landmark_error_4dct_shape():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06765_gb300 as reg
    c = CONFIGS[3]
    p = make_pair(3)
    cfg = reg.make_config(levels=c["levels"], tau=c["eta"], alpha=c["alpha"], mem=c["mem"], max_iter=c["max_iter"],
                          c1=c["c1"])
    r = reg.Registration(cfg)
    t0 = time.perf_counter()
    r.set_images(p["R"], p["T"], p["spacing"])
    u, st = r.register(out="numpy")
    wall = time.perf_counter() - t0
    H = r.level_info(0)["node_spacing"]
    lm_R, lm_T = p["lm_R"], p["lm_T"]
    before = np.linalg.norm(lm_R - lm_T, axis=1)
    after = np.linalg.norm(lm_R + _u_at(u, lm_R, H) - lm_T, axis=1)
    print("landmark error: before %.2f +- %.2f mm, after %.2f +- %.2f mm; registration %.3f s (from host arrays), "
          "iterations %s" % (before.mean(), before.std(), after.mean(), after.std(), wall, st["iters"]))
    assert st["status"] == 0
    assert after.mean() < 0.35 * before.mean()
    r.close()
