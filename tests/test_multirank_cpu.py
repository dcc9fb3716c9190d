"""The multi-GPU bench path's host logic on CPU: two gloo ranks, each with its own batch and time;
the job time is the slowest rank's and the job value counts every rank's batch (weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = [12.5, 40.0][rank]
    ms = bench.reduce_max_ms(dist, my_ms, device="cpu")
    value = bench.weak_scaling_value(world, 1e9, 10, ms)
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_value():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 40.0
    assert value == pytest.approx(2 * 1e9 * 10 / (40.0 * 1e6))


def test_single_process_is_unchanged():
    assert bench.reduce_max_ms(None, 7.0) == 7.0
    assert bench.weak_scaling_value(1, 2e9, 4, 8.0) == pytest.approx(1000.0)
