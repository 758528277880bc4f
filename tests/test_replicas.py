"""Multi-GPU form of the benchmark: independent replicas, one per rank, with the job time
taken as the slowest rank's (no collective on the data path).  The timing reduction is
exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 1000.0 + 250.0 * rank          # rank 1 is the slower one
    ms_max, value = bench.replica_throughput(ms_local, steps=2, n_steps=100, world=world, dist=dist)
    q.put((rank, ms_max, value, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, seed in res:
        assert ms_max == pytest.approx(1250.0)
        # 2 replicas x 2 evaluations x 100 PM steps in 1.25 s
        assert value == pytest.approx(2 * 2 * 100 / 1.25)
    assert res[0][3] != res[1][3]               # each replica simulates its own universe


def test_single_process_throughput_needs_no_process_group():
    ms_max, value = bench.replica_throughput(500.0, steps=3, n_steps=100, world=1)
    assert ms_max == 500.0 and value == pytest.approx(600.0)
