"""bench.py's multi-rank aggregation with two gloo ranks on the CPU: each rank solves its
own RVE (replicas, weak scaling); the job time is the slowest rank's and the work the sum."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, vox = bench.combine_ranks(100.0 + 50.0 * rank, 1e6 * (rank + 1), dist, "cpu")
    out[rank] = (ms, vox)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        assert out[0] == out[1] == (150.0, 3e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 7.0) == (12.5, 7.0)
