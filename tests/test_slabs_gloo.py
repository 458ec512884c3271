"""Host logic of the slab decomposition on CPU ranks (gloo): the partition
of the vertical axis, the neighbour pattern, the halo messages moving
between neighbouring ranks and the FP64 sums of the totals.

Each rank holds its planes of one global array; after the exchange its halo
messages must equal the global array's planes on the far side of its slab
boundaries (two planes deep, the depth of the phi halo), and nothing moves
across the walls at the ends of the axis."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2608_26908_gb300 import slabs  # noqa: E402

NZ, PLANE = 23, 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        glob = np.arange(NZ * PLANE, dtype=np.float64).reshape(NZ, PLANE) * 1.5 - 7.0
        v0, n = slabs.partition(NZ, world)[rank]
        mine = glob[v0:v0 + n]
        send = {slabs.LOWER: torch.tensor(mine[:2].reshape(-1)),
                slabs.UPPER: torch.tensor(mine[-2:].reshape(-1))}
        recv = {s: torch.full((2 * PLANE,), np.nan, dtype=torch.float64) for s in send}
        slabs.exchange(dist, rank, world, send, recv)
        lo, hi = slabs.neighbours(rank, world)
        ok_lo = (np.array_equal(recv[slabs.LOWER].numpy(), glob[v0 - 2:v0].reshape(-1)) if lo is not None
                 else bool(torch.isnan(recv[slabs.LOWER]).all()))
        ok_hi = (np.array_equal(recv[slabs.UPPER].numpy(), glob[v0 + n:v0 + n + 2].reshape(-1))
                 if hi is not None else bool(torch.isnan(recv[slabs.UPPER]).all()))
        # totals: rank r contributes mass r + 1, solute (r, 2r), a solid share
        m, sol, frac = slabs.total(dist, float(rank + 1), [float(rank), 2.0 * rank], 0.25 * rank, n)
        q.put((rank, ok_lo, ok_hi, m, sol.tolist(), frac))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_and_totals_between_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = slabs.partition(NZ, world)
    want_frac = sum(0.25 * r * n for r, (_, n) in enumerate(parts)) / NZ
    for rank, ok_lo, ok_hi, m, sol, frac in out:
        assert ok_lo and ok_hi, rank
        assert m == sum(r + 1 for r in range(world))
        assert sol == [float(sum(range(world))), 2.0 * sum(range(world))]
        assert frac == pytest.approx(want_frac, rel=1e-15)


def test_partition_covers_the_axis_in_order():
    for nz, world in ((23, 2), (23, 3), (64, 8), (4, 2), (17, 5)):
        parts = slabs.partition(nz, world)
        assert parts[0][0] == 0 and sum(n for _, n in parts) == nz
        for (a, n), (b, _) in zip(parts, parts[1:]):
            assert a + n == b
        assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
        assert min(n for _, n in parts) >= 2
    with pytest.raises(ValueError):
        slabs.partition(5, 3)
    assert slabs.neighbours(0, 1) == (None, None)
    assert slabs.neighbours(0, 3) == (None, 1) and slabs.neighbours(2, 3) == (1, None)
