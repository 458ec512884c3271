"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path runs as independent replicas, one per GPU (no data-path exchange):
each rank times its own steps, the job time is the largest rank time, and the
whole-job value counts the cells of every replica.  The reference arm runs on
rank 0 alone; the other ranks return without work.
"""
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


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_setup(None)
        mine = 1.5 + rank  # rank 1 is the slowest
        job = bench.max_over_ranks(mine, dist, "cpu")
        value = bench.job_mlups(w, 1000, 10, job)

        class Args:
            workload, precision, nx, ny, nz, warmup, steps, gpus = "dendrite2d", None, 8, 8, None, 1, 1, 2

        ref_rc = bench.reference_arm(Args) if rank == 1 else None
        q.put((rank, w, r, loc, job, value, ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, w, r, loc, job, value, ref_rc in out:
        assert (w, r, loc) == (2, rank, rank)
        assert job == 2.5  # max over ranks
        assert value == pytest.approx(2 * 1000 * 10 / 2.5 / 1e6)
    assert out[1][6] == 0  # reference arm: rank 1 exits 0 without work


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.job_mlups(1, 2_000_000, 5, 2.0) == pytest.approx(5.0)
