"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the job time is the
maximum over ranks and the value counts the replicas of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [100.0 + 50.0 * rank, 2.0 + rank]           # ms of the timed steps, e2e seconds
    t_ms, e2e_s = bench.max_over_ranks(local, world, "cpu")
    rate = bench.whole_job_rate(1e9, world, t_ms * 1e-3)
    out[rank] = (t_ms, e2e_s, rate)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t_ms, e2e_s, rate = res[rank]
        assert t_ms == 150.0 and e2e_s == 3.0
        # 1e9 attempts per rank, 2 ranks, 0.15 s -> 13.33 attempts/ns
        assert rate == pytest.approx(2e9 / 0.15 / 1e9)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks([1.0, 2.0], 1, "cpu") == [1.0, 2.0]
    assert bench.whole_job_rate(4e9, 1, 2.0) == pytest.approx(2.0)
