"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

With N GPUs every rank registers its own pair (independent replicas, no
collective on the data path); the only cross-rank steps are the barrier around
the timed region and the reductions of the time (max) and of the work (sum).
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    bench.dist_barrier()
    t_max = bench.dist_reduce(10.0 + rank, "max")
    work = bench.dist_reduce(3.0 * (rank + 1), "sum")
    q.put((rank, t_max, work))
    dist.destroy_process_group()


def test_two_rank_reductions():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 11.0, 9.0), (1, 11.0, 9.0)]


def test_single_process_reductions_are_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_reduce(4.5, "max") == 4.5
    assert bench.dist_reduce(4.5, "sum") == 4.5


def test_batch_inputs_pool_matches_serial():
    """The uneven batch generated in a spawn pool equals the serial generation,
    and ranks draw disjoint pair seeds (rank r starts at pair r * n)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    serial = bench.batch_inputs(3, 0, 1)
    pooled = bench.batch_inputs(3, 0, 2)
    for a, b in zip(serial, pooled):
        assert a[2] == b[2] and a[3] == b[3]
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
    other = bench.batch_inputs(1, 3, 1)[0]
    assert other[2] == serial[0][2] and not np.array_equal(other[0], serial[0][0])
