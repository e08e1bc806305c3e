"""Sharded search merge on CPU: world-size-2 gloo ranks each search half of the
configuration space (with the oracle standing in for the GPU search of its
subspace), all-gather their S lowest records and merge them with the library's
bf_merge_lists; the result must equal the oracle's full search."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as dist
    import oracle
    from paper_1904_03621_gb300 import instances, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    o = oracle.get()
    if case == "float":
        J, h = instances.dense_gaussian(16, 8)
        S = 40
    else:
        J, h = instances.dense_pm1(16, 9)
        S = 60
    fb = shard.shard_bits(world)
    en, st = o.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=rank)
    me, ms = shard.gather_and_merge(en, st, S)
    out[rank] = (me.tolist(), [int(x) for x in ms])
    dist.destroy_process_group()


@pytest.mark.parametrize("case", ["float", "int"])
def test_two_rank_merge_equals_full_search(case):
    import torch.multiprocessing as mp
    from paper_1904_03621_gb300 import build
    build.build()
    import oracle
    from paper_1904_03621_gb300 import instances
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    if case == "float":
        J, h = instances.dense_gaussian(16, 8)
        S = 40
    else:
        J, h = instances.dense_pm1(16, 9)
        S = 60
    en_o, st_o = oracle.get().low_spectrum(J, h, S)
    for r in range(2):
        me, ms = out[r]
        assert ms == [int(x) for x in st_o]
        assert np.array_equal(np.array(me), en_o)


def test_merge_lists_host():
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import shard
    a = (np.array([1.0, 3.0, 5.0]), np.array([10, 30, 50], dtype=np.uint64))
    b = (np.array([1.0, 2.0, 3.0]), np.array([11, 20, 29], dtype=np.uint64))
    e, s = shard.merge_lists([a[0], b[0]], [a[1], b[1]], 4)
    assert e.tolist() == [1.0, 1.0, 2.0, 3.0] and s.tolist() == [10, 11, 20, 29]
    with pytest.raises(Exception):
        shard.merge_lists([a[0]], [a[1]], 4)
