"""The multi-rank (weak-scaling) logic of the benchmark, on CPU with the gloo backend.

Instances are independent, so under torchrun every rank runs its own batch and
the only cross-rank steps are the barrier and the max-reduction of the step
time.  This checks those steps with world size 2 (no GPU involved).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = dict(bench.WORKLOADS["kron2-f32-n16"], batch=8)
        b = bench.make_inputs(wl, rank)
        ms = 1.0 + rank            # rank 1 is the slow one
        dist.barrier()
        t = bench.reduce_time_max(ms, dist, torch.device("cpu"))
        digest = torch.tensor([float(np.asarray(b.X, np.float64).sum())], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, digest)
        out[rank] = (t, [g.item() for g in gathered], float(np.asarray(b.A, np.float64).sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_independent_batches():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    t0, g0, a0 = out[0]
    t1, g1, a1 = out[1]
    assert t0 == t1 == 2.0                    # every rank sees the slowest rank's time
    assert g0 == g1 and g0[0] != g0[1]        # each rank drew its own operands
    assert a0 != a1                           # ... and its own components (per-rank seed)


def test_whole_job_rate_is_aggregate():
    assert bench.whole_job_rate(4, 1e9, 1000.0) == pytest.approx(4e9)
    assert bench.rank_seed(1, 0) != bench.rank_seed(1, 1)
