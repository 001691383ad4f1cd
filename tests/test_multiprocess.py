"""Host logic of the N > 1 path on the CPU: two gloo ranks, no GPU.

Problems are sharded by work with no data-path collective; the benchmark's
barrier and max-over-ranks timing run through torch.distributed.
"""
import os
import socket

import pytest

import workload
from paper_1012_2273_gb300.shard import rows_of_worker, shard


def test_paper_row_split_worked_examples():
    # Sec. 3.1.1: 4 rows over 3 workers -> rows {2, 1, 1}, offsets {0, 2, 3}.
    assert [rows_of_worker(4, 3, w) for w in range(3)] == [(0, 2), (2, 1), (3, 1)]
    # Sec. 3.1.2: 4 rows over 2 threads -> {0, 1} and {2, 3}.
    assert [rows_of_worker(4, 2, w) for w in range(2)] == [(0, 2), (2, 2)]
    for rows in (1, 7, 100, 2000):
        for workers in (1, 2, 3, 8):
            parts = [rows_of_worker(rows, workers, w) for w in range(workers)]
            assert sum(c for _, c in parts) == rows
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(workers - 1))


def test_shard_partitions_and_balances():
    sizes = workload.loguniform_sizes(1024, 10, 2000, seed=1)
    for world in (1, 2, 3, 8):
        parts = [shard(sizes, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] ** 3 for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes) ** 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as td

    import bench
    d = bench.Dist()  # gloo on a machine without CUDA
    d.barrier()
    mx = d.max(1.5 + rank)  # per-rank elapsed times: the job time is the slowest rank's
    sizes = workload.loguniform_sizes(64, 10, 2000, seed=1)
    mine = shard(sizes, world, rank)
    gathered = [None] * world
    td.all_gather_object(gathered, mine)
    d.close()
    out.put((rank, mx, gathered))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_barrier_max_and_disjoint_shards():
    import torch
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("the CPU path of Dist (gloo) is what this test covers")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, mx, gathered in results:
        assert mx == 2.5
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(64))
        assert not set(gathered[0]) & set(gathered[1])
