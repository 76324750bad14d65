"""bench.py's host logic on the CPU: the multi-rank aggregation with two gloo ranks (each
rank solves its own RVE: replicas, weak scaling; the job time is the slowest rank's and the
work the sum), and the algorithmic byte model behind the roofline figures."""
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


def _rank_solve(rank, world, port, out):
    """Each rank drives its own solve (the FP64 oracle on a small cell stands in for the
    GPU solve, which needs a device): replicas with different loads, no data-path
    collective; only the timing and work aggregation crosses ranks."""
    import time
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2010_06697_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ph = synth.inclusion_phase(8, 3, 10 + rank, radius=2)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar = np.diag([0.95 - 0.01 * rank, 1.0, 1.0])
    dist.barrier()
    t0 = time.perf_counter()
    r = oracle.admm_solve(ph, par, Fbar, 10.0, 1e-8, 300)
    ms = 1e3 * (time.perf_counter() - t0)
    dist.barrier()
    tot_ms, tot_vox = bench.combine_ranks(ms, ph.size * r["iters"], dist, "cpu")
    out[rank] = (ms, ph.size * r["iters"], tot_ms, tot_vox, r["stress"].tolist(), r["converged"])
    dist.destroy_process_group()


def test_two_gloo_ranks_each_drive_a_solve():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_solve, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0[5] and r1[5]
    # whole-job figures: the slowest rank's time, the sum of the work, the same on both ranks
    assert r0[2] == r1[2] == max(r0[0], r1[0])
    assert r0[3] == r1[3] == r0[1] + r1[1]
    # replicas are independent: each rank's result is its solve alone
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2010_06697_gb300 import synth
    for rank, r in ((0, r0), (1, r1)):
        ph = synth.inclusion_phase(8, 3, 10 + rank, radius=2)
        ref = oracle.admm_solve(ph, synth.two_phase_params(1.0, 10.0), np.diag([0.95 - 0.01 * rank, 1.0, 1.0]),
                                10.0, 1e-8, 300)
        assert np.array_equal(np.array(r[4]), ref["stress"])


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 7.0) == (12.5, 7.0)


def test_byte_model_matches_the_documented_per_voxel_figures():
    """bench.py's algorithmic bytes per voxel and launch (the roofline numerators): one
    iteration of the 3D path in double is 87 s + 1 bytes (s = 8: local 42 s + 1, x-forward
    21 s, four FFT passes 6 s each); the float iteration of the headline takes r_d from the
    spectral solve, so its local pass reads 3 scalars less (39 s + 1) and its z solve also
    reads and writes the kept spectrum (12 s): 90 s + 1 with s = 4.  The double-word polish
    local step moves 301 B, its increment x passes 48 and 48 B (u~ as float pairs)."""
    sys.path.insert(0, ROOT)
    import bench
    it = sum(bench.bytes_per_voxel(c, 8) for c in ("local", "xfwd", "fwd_y", "solve", "inv_y", "xinv"))
    assert it == 87 * 8 + 1
    assert bench.bytes_per_voxel("local", 8) == 42 * 8 + 1 and bench.bytes_per_voxel("xfwd", 8) == 21 * 8
    it = sum(bench.bytes_per_voxel(c, 4) for c in ("local", "xfwd", "fwd_y", "solve", "inv_y", "xinv"))
    assert it == 90 * 4 + 1
    assert bench.bytes_per_voxel("local", 4) == 39 * 4 + 1 and bench.bytes_per_voxel("solve", 4) == 12 * 4
    assert bench.bytes_per_voxel("local_r", 0) == 301
    assert bench.bytes_per_voxel("xfwd_incr", 0) == 48 and bench.bytes_per_voxel("xinv_incr", 0) == 48
    # 2D: d = 2 in the same formulas
    assert bench.bytes_per_voxel("local", 8, d=2) == (4 + 16) * 8 + 1
