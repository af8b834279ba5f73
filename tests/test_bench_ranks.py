"""The multi-rank path of bench.py on CPU: two gloo ranks, no GPU.

With N ranks bench.py runs N independent replicas (the solves shard with no data
exchange) and reports the whole-job rate over the slowest rank's clock.  These
tests run that aggregation over a real world-size-2 process group.
"""
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(seconds[rank], world, torch, torch.device("cpu"))
        q.put((rank, slowest, bench.whole_job_rate(world, 10, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_clock():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds = [0.5, 2.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    results = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in results:
        assert slowest == 2.0
        assert rate == pytest.approx(2 * 10 / 2.0)  # 2 ranks x 10 solves over the slowest rank's 2 s


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.25, 1, torch, torch.device("cpu")) == 0.25
    assert bench.whole_job_rate(1, 8, 0.5) == 16.0


def test_reference_arm_prints_only_on_rank_zero(capsys):
    args = types.SimpleNamespace(nz=128, warmup=0, steps=1, tol=1e-10, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
