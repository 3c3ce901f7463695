"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): each rank
times its own replica of the workload and the job's step time is the maximum
over ranks; rank 0 alone reports."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    got = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    dist.barrier()
    q.put((rank, got))
    dist.destroy_process_group()


def test_step_time_is_the_maximum_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 15.0, 1: 15.0}


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        seed = 0
        workers = 1
        warmup = 1
        steps = 1
        ref_budget = 1.0
        gpus = 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
