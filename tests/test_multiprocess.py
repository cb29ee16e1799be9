"""The N > 1 path of bench.py on CPU: two gloo ranks, whole-job aggregation (maximum of
the times, sum of the work) and the reference arm's rank rule (only rank 0 works)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    times, samples = bench.aggregate([10.0 + rank, 5.0 - rank], 1000 * (rank + 1), world)
    tdist.barrier()
    tdist.destroy_process_group()
    q.put((rank, times, samples))


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, samples in res:
        assert times == [11.0, 5.0]      # max over ranks, per entry
        assert samples == 3000.0         # sum over ranks


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate([1.5, 2.5], 7, 1) == ([1.5, 2.5], 7.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        steps, warmup, storage = 1, 0, "f16"
    bench.run_reference(A())  # returns at once on rank 1: no cube, no oracle, no output
    assert capsys.readouterr().out == ""
