"""The multi-GPU path is replicas only: ranks generate disjoint fields and the
job time is the slowest rank's.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nf = 64
        f0 = bench.replica_field0(rank, nf)
        my_ms = 10.0 + 5.0 * rank  # the slower rank decides
        tot = bench.max_over_ranks(dist, my_ms, "cpu")
        fields = torch.tensor([f0, f0 + nf], dtype=torch.int64)
        gathered = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, fields)
        out[rank] = (tot, [tuple(g.tolist()) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_ranks_disjoint_fields_and_max_time():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        tot, ranges = out[r]
        assert tot == pytest.approx(15.0)
        assert ranges == [(0, 64), (64, 128)]


def test_single_rank_is_identity():
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.replica_field0(0, 64) == 0
