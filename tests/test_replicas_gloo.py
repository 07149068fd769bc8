"""The multi-GPU path of the benchmark, on CPU ranks.

The SWR solve of one problem does not shard across GPUs on one node: `bench.py --gpus N`
runs N replicas (one per rank), takes the slowest rank's time, and reports the units of
all ranks over it.  These tests run that host logic as world-size-2 `gloo` process groups
(no GPU, no collective on the data path)."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.replicas_max_ms(times[rank], "cpu")
        v = bench.whole_job_rate(3.0e8, 2, world, t)
        out.put((rank, t, v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(120.0, 95.0), (40.0, 250.0)])
def test_replicas_take_the_slowest_rank(times):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_replica, args=(r, world, port, times, out))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = max(times)
    for rank, t, v in sorted(res):
        assert t == slow                                   # every rank sees the max
        assert v == pytest.approx(3.0e8 * 2 * world / (slow * 1e-3), rel=1e-15)


def test_single_process_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replicas_max_ms(12.5) == 12.5
    assert bench.whole_job_rate(1e6, 4, 1, 2000.0) == pytest.approx(2e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    def no_work(*a, **k):
        raise AssertionError("a rank other than 0 timed the oracle")

    monkeypatch.setattr(bench, "cpu_oracle_sample", no_work)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = types.SimpleNamespace(impl="reference", gpus=2, steps=1, warmup=0, tc="robin")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
