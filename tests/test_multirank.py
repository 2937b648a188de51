"""Multi-GPU is replicas only (a single system does not shard as the same method): every rank
solves its own replica, the job's time is the slowest rank's, and the reference arm runs on rank
0 alone.  The host logic of that path is checked here with 2 gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    slow = bench.reduce_max(1.5 + rank, "cpu")
    dist.barrier()

    class Args:
        m, prec, cpu_iters, warmup, steps, gpus = 8, "fp64", 1, 0, 1, world

    ref = bench.run_reference(Args) if rank == 1 else None  # rank != 0: no work, exit code 0
    dist.destroy_process_group()
    q.put((rank, w, r, local, slow, ref))


def test_replicas_time_is_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for rank, w, r, local, slow, ref in out:
        assert (w, r, local) == (world, rank, rank)
        assert slow == 2.5
    assert out[1][5] == 0
