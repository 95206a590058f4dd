"""Multi-GPU partition of one molecule's ladder term (host side).

The GPU analogue of the paper's split of the virtual pairs over domains
(Sec. II.D, Eq. pp-Ladder-3): the tensor-core modes evaluate R in tiles of
virtual pairs {a, b} (a in a block of 16, b in a block of 8, a <= b), each
tile the same amount of work; a rank holding B and tau in full computes a
contiguous range of tiles (ladder_set_tile_range), writing R_ij^ab and
R_ij^ba of its pairs only, and the ranks' R, zero elsewhere, add up to the
whole term (one all-reduce), their energies to E_L.  This module holds the
bookkeeping (no arithmetic of the method): the tile enumeration of the
library, balanced ranges, the pairs of a range, and the assembly.
"""
from __future__ import annotations

import numpy as np


def tile_count(v: int) -> int:
    """Pair tiles of a shape: iA over the 16-blocks of a, jB = 2 iA .. vp/8 - 1
    over the 8-blocks of b (vp = v rounded up to 16)."""
    vp = (v + 15) // 16 * 16
    nA, nB8 = vp // 16, vp // 8
    return sum(nB8 - 2 * i for i in range(nA))


def tile_blocks(v: int, tile: int):
    """(iA, jB) of tile number `tile` in the library's a-block-major order."""
    vp = (v + 15) // 16 * 16
    nB8 = vp // 8
    iA, t = 0, tile
    while t >= nB8 - 2 * iA:
        t -= nB8 - 2 * iA
        iA += 1
    return iA, 2 * iA + t


def partition_tiles(ntiles: int, world: int, rank: int):
    """Contiguous range [lo, hi) of tiles for `rank`: every tile costs the
    same, so equal counts balance the work (sizes differ by at most one)."""
    if not (0 <= rank < world) or ntiles < world:
        raise ValueError("need 0 <= rank < world <= ntiles")
    return ntiles * rank // world, ntiles * (rank + 1) // world


def pair_mask(v: int, lo: int, hi: int) -> np.ndarray:
    """Boolean [v, v]: entries (a, b) of R (for every i, j) that tiles
    [lo, hi) write, i.e. both orders of each pair a <= b they own."""
    m = np.zeros((v, v), dtype=bool)
    for tile in range(lo, hi):
        iA, jB = tile_blocks(v, tile)
        diag = (jB >> 1) == iA
        for a in range(16 * iA, min(16 * iA + 16, v)):
            for b in range(8 * jB, min(8 * jB + 8, v)):
                if diag and a > b:
                    continue
                m[a, b] = m[b, a] = True
    return m


def assemble(R, group=None):
    """Sum the ranks' R in place (each rank's R zero outside its tiles) with
    one all-reduce of torch.distributed; the result is the whole term on
    every rank."""
    import torch.distributed as dist
    dist.all_reduce(R, op=dist.ReduceOp.SUM, group=group)
    return R
