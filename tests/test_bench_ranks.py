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


def test_kernel_work_counts_the_algorithmic_bytes():
    """The roofline's numerator.  The tensor-core preconditioner is counted at the scope table's 30 B per
    point per application whatever the launch sequence; its design model beside it: each launch but the
    last moves 4 B per point (FP16 in and out) and the last 8 (FP16 in, the FP16 copy of R, Z in FP32), so
    three launches (frontal slices) move 16 B per point, five (the pair around G fused) 24 and six 28; the
    stencil kernels' per-point bytes are those of their operands."""
    N, dims = 1000, (10, 10, 10)
    amount, unit, bound, worked = bench.kernel_work("modeprod_tc", "fp16", N, dims, 6, 7, 1, 1, 3)
    assert (unit, bound, worked) == ("GB", "hbm", 21)
    assert amount * 1e9 == pytest.approx(7 * 30 * N)
    amount, _, _, worked = bench.kernel_work("modeprod_tc_design", "fp16", N, dims, 6, 7, 1, 1, 3)
    assert worked == 21 and amount * 1e9 == pytest.approx(7 * 16 * N)
    amount, _, _, worked = bench.kernel_work("modeprod_tc_design", "fp16", N, dims, 6, 7, 1, 1, 5)
    assert worked == 35 and amount * 1e9 == pytest.approx(7 * 24 * N)
    amount, _, _, worked = bench.kernel_work("modeprod_tc_design", "fp16", N, dims, 6, 7, 1, 1, 6)
    assert worked == 42 and amount * 1e9 == pytest.approx(7 * 28 * N)
    amount, _, _, worked = bench.kernel_work("modeprod_tc_design", "bf16", N, (10, 10, 1), 6, 7, 1, 1, None)
    assert worked == 28 and amount * 1e9 == pytest.approx(7 * 20 * N)  # 2D, four launches
    amount, _, _, _ = bench.kernel_work("direction", "fp16", N, dims, 6, 7, 1, 1)
    assert amount * 1e9 == pytest.approx(6 * 12 * N)  # Z 4 + P_old 4 in, P 4 out
    amount, _, _, _ = bench.kernel_work("update", "fp16", N, dims, 6, 7, 1, 1)
    assert amount * 1e9 == pytest.approx(6 * 38 * N)  # P 4, R 8+8, U 8+8, FP16 copy 2
    amount, _, _, worked = bench.kernel_work("true_residual", "fp16", N, dims, 6, 7, 1, 2)
    assert worked == 2 and amount * 1e9 == pytest.approx(2 * 26 * N)
    # 4-byte operands (TF32, split BF16 pair): six launches of 8 B per point, the last 12 -> 52 B; the copy
    # of R is 4 B in the update, the check and the initial residual
    amount, _, _, worked = bench.kernel_work("modeprod_tc_design", "bf16x3", N, dims, 3, 4, 1, 1, 6)
    assert worked == 24 and amount * 1e9 == pytest.approx(4 * 52 * N)
    amount, _, _, _ = bench.kernel_work("update", "bf16x3", N, dims, 3, 4, 1, 1)
    assert amount * 1e9 == pytest.approx(3 * 40 * N)
    amount, _, _, _ = bench.kernel_work("true_residual", "tf32", N, dims, 3, 4, 1, 2)
    assert amount * 1e9 == pytest.approx(2 * 28 * N)
    amount, _, _, _ = bench.kernel_work("init_residual", "bf16x3", N, dims, 3, 4, 1, 2)
    assert amount * 1e9 == pytest.approx(1 * 20 * N)
