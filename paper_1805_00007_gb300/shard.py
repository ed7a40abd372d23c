"""Sharding a ragged ensemble over ranks: every instance is an independent problem, so ranks share the
instances and exchange nothing while they step; only per-instance observables are gathered at the end.

One process per GPU (torch.distributed); this module holds the host-side logic only.
"""
from __future__ import annotations


def partition(sizes, world: int) -> list[list[int]]:
    """Instance indices per rank, balanced by lattice nodes: instances in decreasing size, each to the
    rank with the least work so far (ties to the lowest rank, then the lower index).  Deterministic, so
    every rank computes the same assignment without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(ix) for ix in out]


def shard(ensemble, rank: int, world: int):
    """(indices, params, fields) of this rank's share of a list of (params, phi0) instances."""
    sizes = [int(p["nx"]) * int(p["ny"]) for p, _ in ensemble]
    idx = partition(sizes, world)[rank]
    return idx, [ensemble[i][0] for i in idx], [ensemble[i][1] for i in idx]


def gather(values, indices, n_total: int, group=None) -> list:
    """Every rank's per-instance values, placed at their instance indices (an all-gather of Python objects
    over the process group; a list of n_total on every rank)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, list(zip(indices, values)), group=group)
    out = [None] * n_total
    for part in parts:
        for i, v in part:
            out[i] = v
    return out
