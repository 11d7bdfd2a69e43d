"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

BTO needs no communication during an interval (each block is advanced
independently, Sec. 3.1), so the multi-GPU path shards whole blocks across
ranks and only the host-side reporting reduces two numbers at the end. These
tests run that logic with the gloo backend in two spawned processes.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        blocks, ext, org, spc = bench.block_layout(rank, world)
        total, slowest, value = bench.aggregate(1000 * (rank + 1), 0.5 * (rank + 1), world, device="cpu")
        q.put((rank, blocks, org, total, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_blocks_and_aggregate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted([q.get(timeout=120) for _ in range(2)])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    blocks = [set(r[1]) for r in results]
    assert not (blocks[0] & blocks[1])                       # disjoint
    union = blocks[0] | blocks[1]
    assert union == {(bx, by, bz) for bx in range(4) for by in range(2) for bz in range(2)}
    for r in results:
        assert len(r[1]) == 8                                 # same work per rank (weak)
        assert r[3] == 3000.0 and r[4] == 1.0 and r[5] == 3000.0
    # origins follow the block indices at 128 cells of 1/256
    for (bx, by, bz), o in zip(results[1][1], results[1][2]):
        assert o == (bx * 0.5, by * 0.5, bz * 0.5)


def test_single_rank_layout_is_the_256_cube():
    import bench
    blocks, ext, org, spc = bench.block_layout(0, 1)
    assert sorted(blocks) == sorted((bx, by, bz) for bx in range(2) for by in range(2) for bz in range(2))
    assert bench.aggregate(10, 2.0, 1) == (10, 2.0, 5.0)


def test_block_partition_by_work():
    import bench
    from paper_2004_02003_gb300.partition import block_work, partition_blocks
    ext, org, spc, strides = bench.batched_layout()
    work = block_work(ext, strides, 64)
    assert work[0] == 64 * int(np.prod([-(-e // strides[0]) for e in ext[0]]))
    for world in (1, 2, 3, 8):
        parts = partition_blocks(work, world)
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(len(ext)))                 # every block exactly once
        loads = [sum(work[b] for b in p) for p in parts]
        # longest-processing-time rule: within one block of the average
        assert max(loads) - sum(loads) / world <= max(work)
        assert parts == partition_blocks(work, world)         # deterministic
    assert partition_blocks([5, 1], 4)[2:] == [[], []]        # ranks may get nothing


def _partition_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2004_02003_gb300.partition import block_work, partition_blocks
        ext, org, spc, strides = bench.batched_layout()
        mine = partition_blocks(block_work(ext, strides, 64), world)[rank]
        work = sum(block_work([ext[b] for b in mine], [strides[b] for b in mine], 64))
        total, slowest, value = bench.aggregate(work, 1.0 + rank, world, device="cpu")
        q.put((rank, mine, total, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_the_batched_blocks_without_messages():
    import multiprocessing as mp
    import bench
    from paper_2004_02003_gb300.partition import block_work
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted([q.get(timeout=120) for _ in range(2)])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    a, b = set(results[0][1]), set(results[1][1])
    assert not (a & b) and len(a | b) == 512
    ext, org, spc, strides = bench.batched_layout()
    assert results[0][2] == float(sum(block_work(ext, strides, 64))) and results[0][3] == 2.0
