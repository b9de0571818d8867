"""Work partition across ranks (one process per GPU).

k-points are independent (one H, S per k-point, Sec. 2.3), so a batch of
k-points is dealt round-robin to ranks with no data exchange. Within one
k-point the triangle of H and S can be dealt as square tiles in a 2-D
block-cyclic layout over a prow x pcol process grid (the layout a distributed
eigensolver consumes); every rank generates the coefficient columns its tiles
need, so again nothing is exchanged.
"""
from __future__ import annotations

from typing import List, Tuple


def kpoints_of_rank(n_k: int, rank: int, world: int) -> List[int]:
    if world <= 0 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return list(range(rank, n_k, world))


def grid_shape(world: int) -> Tuple[int, int]:
    """Most square prow x pcol grid with prow * pcol == world."""
    p = int(world ** 0.5)
    while world % p:
        p -= 1
    return p, world // p


def owner_of_tile(bi: int, bj: int, prow: int, pcol: int) -> int:
    return (bi % prow) * pcol + (bj % pcol)


def tiles_of_rank(n: int, tile: int, rank: int, world: int, uplo: str = "U") -> List[Tuple[int, int]]:
    """(row block, column block) pairs of the triangle owned by `rank`."""
    prow, pcol = grid_shape(world)
    nb = (n + tile - 1) // tile
    out = []
    for bj in range(nb):
        for bi in range(nb):
            if (uplo == "U" and bi > bj) or (uplo == "L" and bi < bj):
                continue
            if owner_of_tile(bi, bj, prow, pcol) == rank:
                out.append((bi, bj))
    return out
