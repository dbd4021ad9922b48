"""Host logic of the multi-rank bench path on CPU: two gloo ranks on 127.0.0.1.

Every rank solves its own seeded instance of the workload (weak scaling, no collective on
the data path); the reported time is the slowest rank's.
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


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = bench.rank_problem(2, rank, scale=32)          # 32 x 64 sphere
    slowest = bench.max_over_ranks(1.5 + rank, dist)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), D=p.D, Y=p.Yobs, beta=p.beta,
             rowptr=p.graph.rowptr, slowest=slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # same grid and shape, independent data
    assert np.array_equal(r0["rowptr"], r1["rowptr"])
    assert r0["D"].shape == r1["D"].shape and r0["Y"].shape == r1["Y"].shape
    assert not np.allclose(r0["D"], r1["D"])
    assert not np.allclose(r0["beta"], r1["beta"])
    # both ranks report the slowest rank's time
    assert float(r0["slowest"]) == float(r1["slowest"]) == 2.5


def test_rank0_instance_is_the_single_gpu_workload():
    import bench
    import synth
    a = bench.rank_problem(2, 0, scale=32)
    b = synth.config_problem(2, scale=32)
    assert np.array_equal(a.D, b.D) and np.array_equal(a.Yobs, b.Yobs)


def test_blocked_order_applies_to_every_rank():
    import bench
    import synth
    perm = synth.blocked_order(32, 64, 16, 16)
    for rank in (0, 1):
        row = bench.rank_problem(2, rank, scale=32)
        blk = bench.rank_problem(2, rank, scale=32, order="blocked")
        assert np.array_equal(blk.D, row.D[:, perm]) and np.array_equal(blk.Yobs, row.Yobs[:, :, perm])
        assert blk.name == row.name + "_blocked"
