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


SCALE_SORT_MIN = 256


def sort_keys(lengths, last_times=None):
    """(length bucket, time-scale key) of the device's stable sort: lengths up
    to 256 as they are, longer ones in buckets of 32, ordered among
    themselves by the float32 bits of their last breakpoint time when the
    collection has any PCF longer than 256."""
    lengths = np.asarray(lengths, dtype=np.int64)
    hi = np.where(lengths <= SCALE_SORT_MIN, lengths,
                  SCALE_SORT_MIN + ((lengths - SCALE_SORT_MIN) >> 5))
    lo = np.zeros(lengths.size, dtype=np.uint32)
    if last_times is not None and lengths.size and lengths.max() > SCALE_SORT_MIN:
        tl = np.asarray(last_times, dtype=np.float64).astype(np.float32)
        bits = np.where((tl > 0) & np.isfinite(tl), tl, np.float32(0)).view(np.uint32)
        lo = np.where(lengths > SCALE_SORT_MIN, bits, np.uint32(0)).astype(np.uint32)
    return hi, lo


def sorted_order(lengths, last_times=None) -> np.ndarray:
    """Input index of the s-th PCF in the device's sort order (stable)."""
    hi, lo = sort_keys(lengths, last_times)
    return np.lexsort((lo, hi))


TILE_BAND = 16


def tile_order(n: int):
    """(row block, column block) of the pairwise tiles in queue order: column
    blocks from the last (longest PCFs) down in bands of TILE_BAND; inside a
    band, row blocks from the band's last column down to 0, each against the
    band's columns (those >= the row block) from the last down."""
    nb = (n + TILE - 1) // TILE
    out = []
    for c1 in range(nb - 1, -1, -TILE_BAND):
        c0 = max(0, c1 - TILE_BAND + 1)
        for bi in range(c1, -1, -1):
            for bj in range(c1, max(bi, c0) - 1, -1):
                out.append((bi, bj))
    return out


def shard_units(nunits: int, index: int, count: int) -> range:
    if count <= 1:
        return range(nunits)
    if not 0 <= index < count:
        raise ValueError("shard index out of range")
    return range(index, nunits, count)


def shard_pairs(lengths, index: int, count: int, last_times=None):
    """Unordered pairs (i, j), i <= j, in input indices, owned by a shard of
    the tile kernels (``last_times``: each PCF's last breakpoint time, needed
    when some PCF is longer than 256)."""
    n = len(lengths)
    perm = sorted_order(lengths, last_times)
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
