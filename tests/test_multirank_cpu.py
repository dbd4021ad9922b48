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


# ---- batched workload split across ranks ---------------------------------------------------
def _batch_work():
    import synth
    return [s * s * k for s, k in synth.batch_shapes(64)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_batch_partition_covers_every_system_once_and_balances(world):
    from paper_2204_08057_gb300.partition import partition_batch
    work = _batch_work()
    parts = partition_batch(work, world)
    assert len(parts) == world
    flat = sorted(i for q in parts for i in q)
    assert flat == list(range(64))                      # every system exactly once
    loads = [sum(work[i] for i in q) for q in parts]
    # greedy largest-first: the heaviest rank exceeds the mean by less than one system
    assert max(loads) - sum(work) / world < max(work)
    if world <= 4:
        assert max(loads) <= 1.1 * sum(work) / world
    assert parts == partition_batch(work, world)        # every rank computes the same split


def _batch_worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import synth
    from paper_2204_08057_gb300.partition import partition_batch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes = synth.batch_shapes(64)
    mine = partition_batch([s * s * k for s, k in shapes], world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    # a rank builds only its own members, the same problems as in the whole batch
    small = synth.batch_problems(64, side_range=(16, 24), indices=mine[:2])
    full = synth.batch_problems(64, side_range=(16, 24))
    same = all(np.array_equal(a.D, full[i].D) for a, i in zip(small, mine[:2]))
    np.savez(os.path.join(out_dir, f"batch{rank}.npz"), mine=np.array(mine),
             gathered=np.array([len(g) for g in got]), same=same)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_the_batch(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_batch_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = np.load(tmp_path / "batch0.npz")
    r1 = np.load(tmp_path / "batch1.npz")
    a, b = set(r0["mine"].tolist()), set(r1["mine"].tolist())
    assert not (a & b) and a | b == set(range(64))
    work = _batch_work()
    la, lb = sum(work[i] for i in a), sum(work[i] for i in b)
    assert abs(la - lb) < max(work)
    assert list(r0["gathered"]) == list(r1["gathered"]) == [len(a), len(b)]
    assert bool(r0["same"]) and bool(r1["same"])
