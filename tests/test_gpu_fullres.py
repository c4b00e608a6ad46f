"""Parity at full resolution (the volumes the paper's GPU could not hold, Sec. 3.1).

One 512 x 512 x 257 crop of the full-resolution CT workload (0.75 mm): its
finest level has an odd depth, so the deformation grid is not ratio 2 in z
(257 x 257 x 129 nodes for 257 slices) and the multi-pass kernels with the
per-dimension tables of Eq. 3 evaluate it, as on the 1577-slice scans.
Dropping the last slice gives 512 x 512 x 256 with 257 x 257 x 129 nodes,
evaluated by the fused pass.  Each is one evaluation against the FP64 oracle.
"""
import numpy as np
import pytest

from synth import CONFIGS, random_field
from tests.helpers import assert_parity, compare_eval, full_size_node_bound

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fullres_pair():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth.phantoms import make_pair_parallel
    return make_pair_parallel(5, dims=(512, 512, 257))


@pytest.mark.parametrize("depth,impl", [(256, "fused"), (257, "multipass")])
def test_fullres_eval_matches_oracle(fullres_pair, orc, depth, impl):
    import paper_1812_06765_gb300 as reg
    c = CONFIGS[5]
    R = np.ascontiguousarray(fullres_pair["R"][:depth])
    T = np.ascontiguousarray(fullres_pair["T"][:depth])
    dims, h = (512, 512, depth), fullres_pair["spacing"]
    r = reg.Registration(reg.make_config(levels=2, tau=c["eta"], alpha=c["alpha"])).set_images(R, T, h)
    info = r.level_info(0)
    assert info["nodes"] == (257, 257, 129)
    z, tiles = r.level_tiling(0)
    assert (tiles > 0) == (impl == "fused")
    u = random_field(info["nodes"], 1500 + depth, 5.0)
    e = compare_eval(r, orc, R, T, dims, h, u, c["eta"], c["eta"], c["alpha"])
    print(impl, {k: v for k, v in e.items() if k not in ("g", "go")})
    assert_parity(e, node_bound=False)
    full_size_node_bound(e)
    r.close()
