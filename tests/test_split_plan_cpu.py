"""Host logic of the fused pass's z split (no GPU): the load model's plan.

The model: k CTAs per SM, each a slot (k and the tile's output columns ox x oy
come from reg_fused_tile_shape); a tile costs (planes + 7) pipeline steps
times 0.35 + 0.65 x its share of in-image columns (x columns x0-2 .. x0+ox+1
in steps of one, y rows y0-2 .. y0+oy+1); the tiles launch longest segment
group first, then by segment and tile column, each taken by the slot that
frees first.  The replay below is written from that description,
independently of the library's C++."""
import heapq

import pytest

from paper_1812_06765_gb300 import build


@pytest.fixture(scope="module")
def libreg():
    build.build()
    from paper_1812_06765_gb300 import _lib
    return _lib


def _shape():
    from paper_1812_06765_gb300 import _lib
    build.build()
    return _lib.reg_fused_tile_shape()


def _weights(dims):
    ox, oy, _ = _shape()
    mx, my = dims[0], dims[1]
    ntx, nty = -(-mx // ox), -(-my // oy)
    fx = [sum(0 <= x < mx for x in range(ox * t - 2, ox * t + ox + 2)) / (ox + 4) for t in range(ntx)]
    fy = [sum(0 <= y < my for y in range(oy * t - 2, oy * t + oy + 2)) / (oy + 4) for t in range(nty)]
    return [0.35 + 0.65 * fx[tx] * fy[ty] for ty in range(nty) for tx in range(ntx)]


def _makespan(dims, sms, split):
    l1, n1, l2, n2, lr = split
    groups = sorted([(l1, n1, 0), (l2, n2, 1), (lr, 1 if lr else 0, 2)], key=lambda g: (-g[0], g[2]))
    free = [0.0] * (sms * _shape()[2])
    end = 0.0
    for length, count, _ in groups:
        for _ in range(count):
            for w in _weights(dims):
                t = heapq.heappop(free) + w * (length + 7)
                end = max(end, t)
                heapq.heappush(free, t)
    return end


DIMS = [(256, 256, 256), (128, 128, 128), (64, 64, 64), (32, 32, 32), (256, 256, 112), (58, 38, 70), (4, 6, 4)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("sms", [1, 16, 152])
def test_split_plan_covers_the_depth_and_matches_the_model(libreg, dims, sms):
    split, steps = libreg.reg_fused_split_plan(dims, sms)
    l1, n1, l2, n2, lr = split
    assert n1 * l1 + n2 * l2 + lr == dims[2]                 # the segments cover the depth exactly
    assert all(l >= 2 and l % 2 == 0 for l, n in ((l1, n1), (l2, n2)) if n)
    assert lr % 2 == 0 and n1 + n2 + (1 if lr else 0) >= 1
    planes = n1 * (l1 // 2 + 1) + n2 * (l2 // 2 + 1) + (lr // 2 + 1 if lr else 0)
    assert planes <= dims[2] + 2                              # within the tile-partial buffer
    assert steps == pytest.approx(_makespan(dims, sms, split), rel=1e-12)
    # no equal split beats the plan under the same model
    mz = dims[2]
    for k in range(1, mz // 2 + 1):
        tz = 2 * -(-mz // (2 * k))
        uniform = (tz, mz // tz, 0, 0, mz - (mz // tz) * tz)
        assert steps <= _makespan(dims, sms, uniform) + 1e-9


def test_split_plan_at_256_cube_is_uneven(libreg):
    """On 152 SMs the equal splits leave a partial wave; the plan mixes lengths."""
    split, steps = libreg.reg_fused_split_plan((256, 256, 256), 152)
    l1, n1, l2, n2, lr = split
    assert len({l for l, n in ((l1, n1), (l2, n2), (lr, 1 if lr else 0)) if n}) >= 2
    assert steps < _makespan((256, 256, 256), 152, (86, 2, 0, 0, 84))


def test_split_plan_rejects_bad_arguments(libreg):
    for dims, sms in (((255, 256, 256), 152), ((256, 256, 2), 152), ((256, 256, 256), 0)):
        with pytest.raises(libreg.RegError) as ei:
            libreg.reg_fused_split_plan(dims, sms)
        assert ei.value.code == libreg.REG_ERR_ARG
