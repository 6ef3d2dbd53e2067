"""Multi-rank paths on CPU (gloo, world size 2): the bench's max-over-ranks timing and
per-rank input sharding (replicas: no data exchange when halftoning), and the gradient
all-reduce of data-parallel training (the training path's one exchange step)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        import bench
        from paper_2304_12152_gb300 import api
        res = {}
        res["max"] = bench.max_over_ranks(rank + 0.5, world, torch.device("cpu"))
        g = [torch.full((3,), rank + 1.0), torch.full((2, 2), 10.0 * (rank + 1))]
        api.allreduce_grads(g)
        res["g0"] = g[0].tolist()
        res["g1"] = g[1].reshape(-1).tolist()

        class A:
            workload, batch, size, images, side = "printer", 2, 40, 0, 0
        imgs, shapes = bench.build_inputs(A(), rank)
        res["shapes"] = shapes
        res["sum"] = float(sum(float(np.sum(x)) for x in imgs))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_sharding_and_gradient_allreduce():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0["max"] == r1["max"] == 1.5                      # slowest rank's time on every rank
    assert r0["g0"] == r1["g0"] == [1.5, 1.5, 1.5]            # mean gradient on every rank
    assert r0["g1"] == r1["g1"] == [15.0] * 4
    assert r0["shapes"] == r1["shapes"]                       # same per-rank workload (weak scaling) ...
    assert r0["sum"] != r1["sum"]                             # ... on different images


def test_allreduce_without_process_group_is_a_no_op():
    sys.path.insert(0, ROOT)
    from paper_2304_12152_gb300 import api
    g = [torch.ones(4)]
    api.allreduce_grads(g)
    assert g[0].tolist() == [1.0] * 4
