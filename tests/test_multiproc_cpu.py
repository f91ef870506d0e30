"""The N > 1 path of bench.py on CPU: world_size-2 gloo process groups.

bench.py runs one independent replica of the workload per rank (the update
step has no data-path exchange to shard on a single-GPU pool), takes the
slowest rank's time, and reports units of all ranks / that time.  These
tests check that host logic with the gloo backend, and that the reference
arm does its work on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max = bench.max_over_ranks(times[rank], world)
    out.put((rank, t_max, bench.whole_job_rate(512, world, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world, port = 2, _free_port()
    times = [1.5, 2.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t_max, rate in res:
        assert t_max == 2.0
        assert rate == pytest.approx(2 * 512 / 2.0)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(100, 1, 2.0) == 50.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank but 0 exits 0 without work (no oracle run)."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "problem", lambda args: called.append(1))

    class A:
        gpus, steps, warmup, s = 2, 1, 1, 256
    assert bench.main_reference(A()) == 0
    assert not called
