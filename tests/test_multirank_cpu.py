"""The N>1 path of bench.py on CPU: two gloo ranks, one replica each (no
collective on the data path), the job time is the slowest rank's, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # each rank's replica differs (rank seed), same shape
        g = bench.workload(rank)
        sig = torch.tensor([float(g["x"].sum()), float(g["x"].size)], dtype=torch.float64)
        gathered = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, sig)
        # slowest rank's time, whole-job rate
        local_s = 1.0 + rank  # rank 1 is slower
        slowest = bench.max_over_ranks(local_s, dist, torch.device("cpu"))
        rate = bench.job_rate(world, 10, slowest)
        # the reference arm does its work on rank 0 only
        ref_ranks = []
        if rank != 0:
            ref_ranks.append(bench.run_reference(_Args(), rank, world))
        dist.barrier()
        out[rank] = (slowest, rate, [t.tolist() for t in gathered], ref_ranks)
    finally:
        dist.destroy_process_group()


class _Args:
    steps = 1
    warmup = 0


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        slowest, rate, sigs, ref = out[rank]
        assert slowest == 2.0  # max over ranks
        assert rate == pytest.approx(world * 10 / 2.0)
        assert sigs[0][1] == sigs[1][1] and sigs[0][0] != sigs[1][0]  # same size, different replicas
        if rank != 0:
            assert ref == [None]  # no oracle work off rank 0
