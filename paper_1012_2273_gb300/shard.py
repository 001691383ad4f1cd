"""Sharding independent products across ranks (one process per GPU).

The products of a grouped call are independent, so a batch splits across GPUs
with no data exchange: each rank runs mm_gemm_grouped on its own share.  The
paper splits rows of one product across workers instead (Alg. 2-4, remainder
rows to the first workers); here whole problems are dealt out by estimated
work, longest first (LPT), which keeps the ranks within one problem of each
other.
"""
from __future__ import annotations

import heapq


def shard(sizes: list[int], world: int, rank: int) -> list[int]:
    """Indices of the problems rank `rank` of `world` computes (work ~ N^3)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    loads = [(0, r) for r in range(world)]
    heapq.heapify(loads)
    mine = []
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        load, r = heapq.heappop(loads)
        if r == rank:
            mine.append(i)
        heapq.heappush(loads, (load + sizes[i] ** 3, r))
    return sorted(mine)


def rows_of_worker(rows: int, workers: int, worker: int) -> tuple[int, int]:
    """The paper's row split (Sec. 3.1.1, Alg. 2): `rows // workers` each, the
    remainder one extra to each of the first workers.  Returns (offset, count)
    for worker index `worker` (0-based)."""
    ave, extra = divmod(rows, workers)
    count = ave + (1 if worker < extra else 0)
    offset = worker * ave + min(worker, extra)
    return offset, count
