"""Splitting one pairwise matrix across GPUs (one process per GPU).

Every pair is independent (Sec. 3.1: the matrix is N^2 separate integrals), so
a matrix is split by work unit with no data exchange during the walk: rank r
of W computes the 32 x 32 tiles (merge path: the pairs) u of the kernel's
queue order with u % W == r and writes only their entries; the partial
matrices are then summed (entries outside a shard stay 0) or kept sharded.
The paper spreads block rows over GPUs with work stealing (Sec. 6); strided
ownership of the longest-first tile order balances the load statically.

The host-side functions here mirror the device's length sort and tile order
so that the ownership of every pair can be enumerated without a GPU.
"""
from __future__ import annotations

import numpy as np

TILE = 32


def sorted_order(lengths) -> np.ndarray:
    """Input index of the s-th shortest PCF (stable, as the device sort)."""
    return np.argsort(np.asarray(lengths), kind="stable")


def tile_order(n: int):
    """(row block, column block) of the pairwise tiles in queue order:
    column blocks from the last (longest PCFs) down, rows bi = bj .. 0."""
    nb = (n + TILE - 1) // TILE
    out = []
    for bj in range(nb - 1, -1, -1):
        for bi in range(bj, -1, -1):
            out.append((bi, bj))
    return out


def shard_units(nunits: int, index: int, count: int) -> range:
    if count <= 1:
        return range(nunits)
    if not 0 <= index < count:
        raise ValueError("shard index out of range")
    return range(index, nunits, count)


def shard_pairs(lengths, index: int, count: int):
    """Unordered pairs (i, j), i <= j, in input indices, owned by a shard of
    the tile kernels."""
    n = len(lengths)
    perm = sorted_order(lengths)
    tiles = tile_order(n)
    owned = set()
    for u in shard_units(len(tiles), index, count):
        bi, bj = tiles[u]
        rows = perm[bi * TILE: min(n, (bi + 1) * TILE)]
        cols = perm[bj * TILE: min(n, (bj + 1) * TILE)]
        for r in rows:
            for c in cols:
                owned.add((min(int(r), int(c)), max(int(r), int(c))))
    return owned


def pairwise_shard(x, metrics, rank: int, world: int, precision="f32c", out_dtype=None,
                   schedule="tile1024", **kw):
    """This rank's part of the pairwise matrices: N x N tensors holding the
    entries of the owned tiles (both triangles) and zeros elsewhere.  All
    ranks must use the same schedule kernel."""
    import torch

    from . import api
    out_dtype = out_dtype or torch.float32
    n = x.n
    outs = [torch.zeros((n, n), dtype=out_dtype, device=x.times.device) for _ in metrics]
    api.pcf_pairwise(x, metrics, precision=precision, out=outs, schedule=schedule,
                     shard=(rank, world), **kw)
    return outs
