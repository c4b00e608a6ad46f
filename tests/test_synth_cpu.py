"""Input generators: the slab-parallel generation of the full-resolution CT
workload gives exactly the serial arrays (any split of the planes draws the
same per-slab noise)."""
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
