"""Two-rank runs of the benchmark's multi-GPU path on CPU (gloo).

With --gpus N every rank advances its own ensemble members (seeds 1000 apart per
rank); the job's time is the slowest rank's and its work the sum over ranks, with
no collective on the data path.  Here each rank steps its member with the oracle
(a CPU stand-in for its GPU) through the bench's own seeding, stepping and
aggregation functions, and the parent checks the aggregate against the ranks'
own figures and a serial re-run of each rank's member."""
import os
import socket

import torch.multiprocessing as mp

JMIN, JMAX, EPS, STEPS = 2, 3, 1e-2, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(target, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


def _rank_scalars(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds, cells = bench.combine_ranks(1.5 + rank, 100.0 * (rank + 1), "cpu", world)
    out.put((rank, seconds, cells))
    dist.barrier()
    dist.destroy_process_group()


def _rank_member(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import grid
    hy = grid.Hierarchy(JMIN, JMAX)
    seed = bench.member_seeds(0, rank, 1)[0]
    M = bench.oracle_member(hy, EPS, seed, JMAX)
    cells, secs = bench.oracle_steps(M, STEPS)
    job_secs, job_cells = bench.combine_ranks(secs, cells, "cpu", world)
    out.put((rank, seed, cells, secs, job_secs, job_cells, M.mass(), float(M.dh[JMIN].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_two_ranks():
    assert _spawn(_rank_scalars, 2) == [(0, 2.5, 300.0), (1, 2.5, 300.0)]


def test_combine_one_rank():
    import bench
    assert bench.combine_ranks(1.25, 7.0, "cpu", 1) == (1.25, 7.0)


def test_member_seeds():
    import bench
    assert bench.member_seeds(0, 0, 3) == [0, 1, 2]
    assert bench.member_seeds(5, 2, 2) == [2005, 2006]


def test_two_ranks_step_their_own_members():
    import bench
    from oracle import grid
    got = _spawn(_rank_member, 2)
    seeds = [g[1] for g in got]
    assert seeds == [0, 1000]
    # the whole-job figures: slowest rank's time, sum of the ranks' cells, on every rank
    for g in got:
        assert g[4] == max(x[3] for x in got)
        assert g[5] == sum(x[2] for x in got)
    # each rank advanced the member of its own seed: a serial re-run gives the same
    # cells, mass and depth, and the two ranks' members differ
    hy = grid.Hierarchy(JMIN, JMAX)
    for rank, seed, cells, _, _, _, mass, dsum in got:
        M = bench.oracle_member(hy, EPS, seed, JMAX)
        c, _ = bench.oracle_steps(M, STEPS)
        assert (c, M.mass(), float(M.dh[JMIN].sum())) == (cells, mass, dsum)
    assert got[0][7] != got[1][7]
