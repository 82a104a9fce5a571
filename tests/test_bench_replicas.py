"""The multi-GPU path of bench.py is independent replicas ("replicas only":
the method has no exchange step on one box): every rank runs its own
solve, the job's step time is the slowest rank's, and value = step time /
world per solve.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    ms = bench.max_over_ranks(step_ms, dist, "cpu")
    out[rank] = (ms, bench.seconds_per_solve(ms, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, per_solve = out[r]
        assert ms == 150.0
        assert per_solve == pytest.approx(0.075)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.seconds_per_solve(2000.0, 1) == 2.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle) runs once: ranks other
    than 0 return at once and print nothing."""
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 0

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
