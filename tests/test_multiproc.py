"""The N > 1 path of bench.py (replicas, no data-path collective): gloo
barrier and max-over-ranks timing with world size 2 on CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # each replica's own timing; the job's time is the slowest rank's
    mine = 1.0 + rank
    q.put((rank, bench.all_max(w, mine)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 2.0, 1: 2.0}


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    import bench

    class A:
        workload = "1024x1024_k7"
        steps = 2
        warmup = 1
        gpus = 2

    bench.run_reference(A, world=2, rank=1)
    assert capsys.readouterr().out == ""
