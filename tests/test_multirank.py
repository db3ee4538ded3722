"""The N > 1 benchmark path on CPU: two gloo ranks (replicas only, no data
path collective) agree on the slowest rank's time and on the whole-job rate;
the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    slow = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(600, world, slow)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slow, rate))


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate in out:
        assert slow == 20.0
        assert abs(rate - 600 * 2 / 0.020) < 1e-6


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    # rank 1 returns at once: no oracle, no output
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=2)) is None
