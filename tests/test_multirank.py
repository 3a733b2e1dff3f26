"""The bench's multi-rank aggregation on CPU (gloo, world size 2): every rank runs a replica of
the workload, the job's time is the slowest rank's and the job's rate counts every rank's
units (the path has no data-path collective: replicas only)."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" (r + 1) x 10 ms per step and (r + 1) x 3 ms to build
    got = bench.max_over_ranks([10.0 * (rank + 1), 3.0 * (rank + 1)], dist, "cpu")
    rate = bench.job_rate(1000.0, world, got[0] / 1e3)
    out.put((rank, got, rate, bench._dist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_both():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate, env in res:
        assert got == [20.0, 6.0]                    # the slower replica's times on every rank
        assert rate == pytest.approx(1000.0 * 2 / 0.020)
        assert env[0] == 2 and env[1] == rank        # WORLD_SIZE, RANK as torchrun sets them


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
