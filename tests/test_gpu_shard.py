"""The sharded search's GPU path on one device: every rank's share (shard.search_shard, the
library calls of shard.sharded_low_spectrum) runs in turn on this GPU, the shares are merged
with bf_merge_lists and the result is compared with the oracle's full search.  Power-of-two and
other world sizes (contiguous chunk ranges) are covered."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from parity import assert_float_parity, assert_int_equal
from paper_1904_03621_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    return api


def merged(J, h, S, world):
    import torch
    from paper_1904_03621_gb300 import shard
    Jd, hd = torch.as_tensor(J).cuda(), torch.as_tensor(h).cuda()
    shares = [shard.pad_list(*shard.search_shard(Jd, hd, S, r, world), S) for r in range(world)]
    return shard.merge_lists([e for e, _ in shares], [c for _, c in shares], S)


@pytest.mark.parametrize("world", [2, 3, 4, 5, 7])
def test_shards_on_one_gpu_equal_full_search(bf, world):
    o = oracle.get()
    J, h = instances.dense_gaussian(24, 900 + world)
    en, st = merged(J, h, 200, world)
    en_o, st_o = o.low_spectrum(J, h, 201)
    assert_float_parity(o, J, h, en, st, en_o, st_o)
    Ji, hi = instances.dense_pm1(22, 910 + world)
    en, st = merged(Ji, hi, 300, world)
    en_o, st_o = o.low_spectrum(Ji, hi, 300)
    assert_int_equal(en, st, en_o, st_o)


def test_shards_small_space(bf):
    """A space too small to split among the ranks (2^8 configurations, S = 200): one rank searches
    it all and the others contribute padding only."""
    o = oracle.get()
    J, h = instances.dense_pm1(8, 920)
    en, st = merged(J, h, 200, 3)
    en_o, st_o = o.low_spectrum(J, h, 200)
    assert_int_equal(en, st, en_o, st_o)
