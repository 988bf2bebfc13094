"""The multi-rank path of bench.py on CPU: two gloo ranks (one process each) shard the channels
(each rank draws its own, no data crosses ranks), agree on the slowest rank's time, and report
the whole-job rate over all ranks. The detector runs on one GPU per rank; the rank logic around
it needs no GPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch, w = bench.load_batch(0.002, rank, "rayleigh_32x32_64qam")
        digest = torch.tensor([float(np.abs(batch.H).sum()), float(batch.n_channels)],
                              dtype=torch.float64)
        got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(got, digest)
        my_ms = 10.0 + 5.0 * rank
        ms = bench.max_over_ranks(my_ms, dist)
        rate = bench.whole_job_rate(batch.n_channels * w["chains"] * w["iterations"], world,
                                    ms * 1e-3)
        out[rank] = (ms, rate, [tuple(g.tolist()) for g in got])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_agree():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    ms0, rate0, got0 = out[0]
    ms1, rate1, got1 = out[1]
    assert ms0 == ms1 == 15.0                       # both ranks report the slowest rank's time
    assert rate0 == rate1
    assert got0 == got1
    (s0, n0), (s1, n1) = got0
    assert n0 == n1 > 0 and s0 != s1                # same shape of work, different channels
    import bench
    w = bench.workload.WORKLOADS["rayleigh_32x32_64qam"]
    assert rate0 == pytest.approx(n0 * w["chains"] * w["iterations"] * 2 / 15e-3)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.rank_seed(1002, 0) == 1002 and bench.rank_seed(1002, 3) != 1002
