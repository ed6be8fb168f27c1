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


def test_clock_sampler_summary(tmp_path, monkeypatch):
    """The clock summary of the bench line: median and maximum SM clock and every
    active throttle reason but idle, from nvidia-smi's CSV (here a stand-in script)."""
    import time
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '1980, 2070, 1200.5, 0x0000000000000004'\n"
                    "echo '2070, 2070, 1300.0, 0x0000000000000001'\n"
                    "echo '2070, 2070, 1310.0, 0x0000000000000028'\n"
                    "echo 'N/A, N/A, N/A, N/A'\n"
                    "sleep 5\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    monkeypatch.delenv("MUCA_CLOCKS_CSV", raising=False)
    c = bench.ClockSampler(0)
    c.start()
    for _ in range(50):
        if os.path.exists(c.path) and os.path.getsize(c.path) > 100:
            break
        time.sleep(0.05)
    r = c.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3,
                 "reasons": ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]}
    assert not os.path.exists(c.path)  # temporary samples are removed
