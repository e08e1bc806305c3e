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


def rank_subspaces(rank: int, world: int, n: int, S: int):
    """Subspaces (fixed_bits, fixed_value) that rank `rank` of `world` searches.

    The top `cb` configuration bits split the space into 2^cb chunks (Eq. (6)); rank r takes
    the contiguous chunk range [r 2^cb / world, (r+1) 2^cb / world), written as the fewest
    aligned blocks (each block is one subspace with fewer fixed bits).  A power-of-two world
    gets one subspace per rank (cb = log2 world); any other world uses cb = ceil(log2 world) + 4,
    so the ranks' shares differ by at most one chunk in 16 per rank.  cb is capped so that every
    subspace still holds at least S configurations.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    if world & (world - 1) == 0:
        cb = world.bit_length() - 1
    else:
        cb = (world - 1).bit_length() + 4
    cap = n - max(int(S - 1).bit_length(), 0)
    cb = min(cb, max(cap, 0), n)
    chunks = 1 << cb
    lo, hi = rank * chunks // world, (rank + 1) * chunks // world
    out = []
    while lo < hi:
        k = 0
        while k < cb and lo % (1 << (k + 1)) == 0 and lo + (1 << (k + 1)) <= hi:
            k += 1
        out.append((cb - k, lo >> k))
        lo += 1 << k
    return out


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


def search_shard(J, h, S: int, rank: int, world: int, **kw):
    """This rank's share of one search (CUDA tensors J, h): one library call per subspace of
    rank_subspaces, merged on the host.  Returns (energies, states) as numpy arrays with S
    records, or fewer when the share holds fewer than S configurations."""
    import torch
    from . import api
    n = J.shape[0]
    lists_e, lists_s = [], []
    if not rank_subspaces(rank, world, n, S):          # a small space: other ranks hold all of it
        return np.empty(0, dtype=np.int64 if J.dtype == torch.int32 else np.float64), np.empty(0, dtype=np.uint64)
    for fb, fv in rank_subspaces(rank, world, n, S):
        k = min(S, 1 << (n - fb))
        en, st = api.low_spectrum(J, h, k, fixed_bits=fb, fixed_value=fv, **kw) if fb else \
            api.low_spectrum(J, h, k, **kw)
        lists_e.append(en.cpu().numpy())
        lists_s.append(api.states_u64(st))
    if len(lists_e) == 1:
        return lists_e[0], lists_s[0]
    L = max(len(e) for e in lists_e)
    pe, ps = zip(*(pad_list(e, c, L) for e, c in zip(lists_e, lists_s)))
    total = sum(len(e) for e in lists_e)
    return merge_lists(list(pe), list(ps), min(S, total))


def pad_list(energies, states, length: int):
    """Pad a sorted (energies, states) list to `length` with records that sort after every real one
    (the host merge takes lists of equal length)."""
    is_int = np.issubdtype(np.asarray(energies).dtype, np.integer)
    e = np.asarray(energies, dtype=np.int64 if is_int else np.float64)
    c = np.asarray(states, dtype=np.uint64)
    k = length - len(e)
    big = np.iinfo(np.int64).max if is_int else np.inf
    return (np.concatenate([e, np.full(k, big, dtype=e.dtype)]),
            np.concatenate([c, np.full(k, np.iinfo(np.uint64).max, dtype=np.uint64)]))


def sharded_low_spectrum(J, h, S: int, group=None, **kw):
    """One instance searched by all ranks of `group` (CUDA tensors J, h on this rank's GPU).

    Rank r searches the subspaces of rank_subspaces(r, world, n, S); returns the merged
    (energies, states) as numpy arrays on every rank.
    """
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    en, st = search_shard(J, h, S, rank, world, **kw)
    en, st = pad_list(en, st, S)      # a share smaller than S configurations
    return gather_and_merge(en, st, S, group)
