"""The N > 1 host path of bench.py on CPU: two gloo ranks (world size 2).

bench.py under torchrun runs one independent solve per GPU (weak scaling, no
data-path collective); the only cross-rank steps are the barriers around the
timed region, the max-over-ranks of the elapsed time and the broadcast of
rank 0's Schwarz block choice, exercised here.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(world, 1.0 + rank, device="cpu")
    c = bench.from_rank0(world, 7 + rank, device="cpu")  # the block choice every replica runs
    bench.barrier(world)
    q.put((rank, (t, c)))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: (2.0, 7), 1: (2.0, 7)}


def test_reference_arm_silent_on_nonzero_rank(monkeypatch, capsys):
    import bench

    class A:
        steps, warmup, gpus, gpu_iterations = 1, 0, 2, 7
        workload = bench.WORKLOAD

    assert bench.run_reference(A, world=2, rank=1) == 0
    assert capsys.readouterr().out == ""
