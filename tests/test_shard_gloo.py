"""Sharded search merge on CPU: gloo ranks (world size 2, and 3 for the
non-power-of-two split) each search their share of the configuration space (with
the oracle standing in for the GPU search of each subspace), all-gather their S
lowest records and merge them with the library's bf_merge_lists; the result must
equal the oracle's full search."""
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
    # the rank's subspaces (one for a power-of-two world, contiguous chunk ranges otherwise)
    lists = [o.low_spectrum(J, h, min(S, 1 << (16 - fb)), fixed_bits=fb, fixed_value=fv)
             for fb, fv in shard.rank_subspaces(rank, world, 16, S)]
    L = max(len(e) for e, _ in lists)
    padded = [shard.pad_list(e, c, L) for e, c in lists]
    en, st = shard.merge_lists([p[0] for p in padded], [p[1] for p in padded], min(S, sum(len(e) for e, _ in lists)))
    en, st = shard.pad_list(en, st, S)
    me, ms = shard.gather_and_merge(en, st, S)
    out[rank] = (me.tolist(), [int(x) for x in ms])
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("float", 2), ("int", 2), ("float", 3)])
def test_rank_merge_equals_full_search(case, world):
    import torch.multiprocessing as mp
    from paper_1904_03621_gb300 import build
    build.build()
    import oracle
    from paper_1904_03621_gb300 import instances
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, out)) for r in range(world)]
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
    for r in range(world):
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


def test_rank_subspaces_partition_the_space():
    """For every world size the ranks' subspaces tile [0, 2^n) exactly, with shares within one chunk."""
    from paper_1904_03621_gb300.shard import rank_subspaces
    for n, S in ((20, 10), (30, 1000), (12, 100)):
        for world in range(1, 13):
            cover = []
            for r in range(world):
                for fb, fv in rank_subspaces(r, world, n, S):
                    assert (1 << (n - fb)) >= S
                    lo = fv << (n - fb)
                    cover.append((lo, lo + (1 << (n - fb)), r))
            cover.sort()
            assert cover[0][0] == 0 and cover[-1][1] == 1 << n
            assert all(a[1] == b[0] for a, b in zip(cover, cover[1:]))
            if world & (world - 1) == 0 and (1 << n) // world >= S:
                assert all(len(rank_subspaces(r, world, n, S)) == 1 for r in range(world))
