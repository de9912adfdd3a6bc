"""Host logic of bench.py's multi-process path on CPU (gloo, world size 2).

With N GPUs each rank runs an independent replica of the workload (the hot
path has no data exchange between GPUs); the ranks meet at a
barrier around the timed region and rank 0 reports the maximum time.
"""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(world)
    t = 1.0 + rank  # per-rank step time
    out[rank] = bench.reduce_max(t, world)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_rank_replicas_report_max_time():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 2.0


def test_single_process_defaults():
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.reduce_max(3.5, 1) == 3.5
