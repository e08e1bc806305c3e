"""Splitting one search across processes (one GPU each) and merging the results.

The configuration space splits into disjoint subspaces by fixing the top
bits of c (the chunk offset of the paper's Sec. 3, Eq. (6)); each rank searches
its own subspace and the S lowest records overall are the S lowest of the
union of the per-rank lists (one all-gather of S records per rank, then
bf_merge_lists on the host).  No collective touches the enumeration itself.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def shard_bits(world: int) -> int:
    """Number of fixed top bits for `world` shards (world must be a power of two)."""
    if world < 1 or world & (world - 1):
        raise ValueError("the number of shards must be a power of two")
    return world.bit_length() - 1


def merge_lists(energy_lists, state_lists, S: int):
    """S lowest records of several (energies, states) lists (numpy arrays, host)."""
    lib = _lib.load()
    k = len(energy_lists)
    is_int = np.issubdtype(np.asarray(energy_lists[0]).dtype, np.integer)
    en = [np.ascontiguousarray(e, dtype=np.int64 if is_int else np.float64) for e in energy_lists]
    st = [np.ascontiguousarray(s, dtype=np.uint64) for s in state_lists]
    S_each = en[0].shape[0]
    if any(e.shape[0] != S_each for e in en) or any(s.shape[0] != S_each for s in st):
        raise ValueError("all lists must have the same length")
    ep = (ctypes.c_void_p * k)(*[e.ctypes.data for e in en])
    sp = (ctypes.c_void_p * k)(*[s.ctypes.data for s in st])
    out_e = np.empty(S, dtype=np.int64 if is_int else np.float64)
    out_s = np.empty(S, dtype=np.uint64)
    status = lib.bf_merge_lists(k, ep, sp, S_each, _lib.BF_I32 if is_int else _lib.BF_F64, S,
                                out_e.ctypes.data, out_s.ctypes.data)
    _lib.check(status, lib)
    return out_e, out_s


def gather_and_merge(energies, states, S: int, group=None):
    """All-gather every rank's (energies, states) (numpy, length S) and merge them."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    is_int = np.issubdtype(np.asarray(energies).dtype, np.integer)
    e = torch.from_numpy(np.ascontiguousarray(energies, dtype=np.int64 if is_int else np.float64))
    s = torch.from_numpy(np.ascontiguousarray(states, dtype=np.uint64).view(np.int64))
    es = [torch.empty_like(e) for _ in range(world)]
    ss = [torch.empty_like(s) for _ in range(world)]
    dist.all_gather(es, e, group=group)
    dist.all_gather(ss, s, group=group)
    return merge_lists([x.numpy() for x in es], [x.numpy().view(np.uint64) for x in ss], S)


def sharded_low_spectrum(J, h, S: int, group=None, **kw):
    """One instance searched by all ranks of `group` (CUDA tensors J, h on this rank's GPU).

    Rank r searches the subspace whose top log2(world) bits equal r; returns the merged
    (energies, states) as numpy arrays on every rank.
    """
    import torch.distributed as dist
    from . import api
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    fb = shard_bits(world)
    en, st = api.low_spectrum(J, h, S, fixed_bits=fb, fixed_value=rank, **kw) if fb else api.low_spectrum(J, h, S, **kw)
    return gather_and_merge(en.cpu().numpy(), api.states_u64(st), S, group)
