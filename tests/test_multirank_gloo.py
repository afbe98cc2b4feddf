"""N > 1 host path on CPU: two gloo ranks, independent problems, aggregation."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        from paper_2202_02847_gb300 import multirank, workloads as W
        from paper_2202_02847_gb300.fmm import UniformPass
        import __graft_entry__  # noqa: F401
        tree = W.uniform_octree(3, 4096, seed=multirank.rank_seed(2, rank))
        fp = UniformPass(tree, 4, None, device="cpu")
        units = fp.counts["m2l"]
        secs = 1.0 + rank                       # rank 1 is the slow one
        rate, tmax = multirank.aggregate_rate(units, secs)
        digest = float(np.abs(tree.points).sum())
        d = torch.tensor([digest], dtype=torch.float64)
        all_d = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(all_d, d)
        out[rank] = (rate, tmax, units, [float(x) for x in all_d])
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    import __graft_entry__
    __graft_entry__.build_library()
    world = 2
    mgr = mp.get_context("spawn").Manager()      # no fork of this (threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    units = r0[2]
    assert r1[2] == units                       # same workload shape per rank
    assert r0[1] == r1[1] == 2.0                # max over ranks
    assert r0[0] == pytest.approx(2 * units / 2.0)
    assert r0[3][0] != r0[3][1]                 # independent problems (different seeds)


def test_single_process_aggregate():
    from paper_2202_02847_gb300 import multirank
    assert multirank.aggregate_rate(100, 2.0) == (50.0, 2.0)
