"""Two-rank run of the benchmark's whole-job aggregation on CPU (gloo).

With --gpus N every rank advances its own ensemble member; the job's time is the
slowest rank's and its work the sum over ranks (no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds, cells = bench.combine_ranks(1.5 + rank, 100.0 * (rank + 1), "cpu", world)
    out.put((rank, seconds, cells))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2.5, 300.0), (1, 2.5, 300.0)]


def test_combine_one_rank():
    import bench
    assert bench.combine_ranks(1.25, 7.0, "cpu", 1) == (1.25, 7.0)
