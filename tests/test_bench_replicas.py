"""CPU test of the multi-GPU replica logic of bench.py with two gloo ranks.

bench.py --gpus N runs one independent replica of the workload per GPU (the
solve does not shard across GPUs on this pool); its only cross-rank step is the
max over ranks of the timed region, and the whole-job value counts the solves
of every rank.  Both are exercised here on the CPU with world_size 2.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # the slower rank decides the step time
    m = bench.reduce_max(ms, dist, device="cpu")
    out[rank] = (m, bench.replica_value(2, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 150.0
    # 2 solves per step on each of 2 ranks in 150 ms
    assert abs(out[0][1] - 4 / 0.150) < 1e-9


def test_single_rank_helpers():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert abs(bench.replica_value(2, 1, 250.0) - 8.0) < 1e-12
