"""The multi-GPU path of bench.py (independent replicas, weak scaling) on two
CPU ranks over gloo: the whole-job figures take each shape's slowest replica
and scale the geo-mean by the number of replicas."""
import os
import socket
import tempfile

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        flops = np.array([2e9, 8e9, 3e10])
        med = np.array([0.010, 0.020, 0.050]) * (1.0 + 0.5 * rank)   # rank 1 slower
        total_ms = 7.0 + rank

        def all_reduce_max(arr):
            t = torch.tensor(arr, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return t.numpy()

        got_med, got_total, value = bench.aggregate_replicas(med, total_ms, flops, world,
                                                             all_reduce_max)
        if rank == 0:
            np.save(out_path, np.append(got_med, [got_total, value]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_and_scale():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "agg.npy")
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = np.load(out)
    med, total, value = res[:3], res[3], res[4]
    slow = np.array([0.010, 0.020, 0.050]) * 1.5
    assert np.allclose(med, slow) and total == 8.0
    flops = np.array([2e9, 8e9, 3e10])
    want = float(np.exp(np.mean(np.log(flops / (slow * 1e-3) / 1e12)))) * world
    assert abs(value - want) < 1e-9 * want


def test_single_replica_is_unchanged():
    flops = np.array([1e9, 4e9])
    med = np.array([0.01, 0.02])
    got_med, total, value = bench.aggregate_replicas(med, 3.0, flops, 1)
    assert np.array_equal(got_med, med) and total == 3.0
    assert abs(value - bench.geomean(flops / (med * 1e-3) / 1e12)) < 1e-12
