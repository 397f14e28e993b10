"""The multi-rank path of bench.py on CPU with gloo, world size 2: ranks
search disjoint trees (no data-path collective) and the job time of a phase
is the slowest rank's."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ids = bench.shard_tree_ids(rank, 4096)
    seconds = 1.5 + rank            # rank 1 is the slow one
    job = bench.max_over_ranks(seconds, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, (int(ids[0]), int(ids[-1]), bench.root_seed_of(rank, 2)))
    if rank == 0:
        out.put((job, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    job, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert job == 2.5
    (a0, a1, s0), (b0, b1, s1) = gathered
    assert (a0, a1) == (0, 4095) and (b0, b1) == (4096, 8191)   # disjoint stream ids
    assert s0 != s1                                             # each rank its own roots


def test_shards_cover_without_overlap():
    import bench
    ids = np.concatenate([bench.shard_tree_ids(r, 100) for r in range(8)])
    assert len(np.unique(ids)) == 800 and ids.min() == 0 and ids.max() == 799
