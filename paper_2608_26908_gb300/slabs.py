"""Slab decomposition of a 3D grid along its vertical axis, one slab per
rank (the paper runs its solver as a CPU domain decomposition, Appendix A;
here each slab is a library handle, gpflbm_create_slab, on its own GPU).

Per step every slab packs the planes its neighbours need into device
messages (gpflbm_halo_pack), the messages move between neighbouring ranks
(torch.distributed point-to-point: NCCL between GPUs, gloo on CPU), each
slab unpacks what it received into its halo planes (gpflbm_halo_unpack) and
steps once.  The conservation totals are summed over the ranks in FP64.
Nothing else is exchanged: the step is local once the halo planes hold the
neighbours' values.

This module holds the host logic only (the partition, the neighbour
pattern, the transfers and the sums); the arithmetic runs in the library.
"""
import numpy as np

LOWER, UPPER = 0, 1


def partition(nz, world, minimum=2):
    """(v_begin, v_count) of each rank's slab: contiguous, as even as the
    planes allow, every slab at least `minimum` planes (the halo is two
    planes of phi deep)."""
    if world < 1 or nz < minimum * world:
        raise ValueError("%d planes cannot give %d slabs of at least %d planes" % (nz, world, minimum))
    base, extra = divmod(nz, world)
    out, v = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((v, n))
        v += n
    return out


def neighbours(rank, world):
    """(rank below, rank above), None at a wall of the vertical axis."""
    return (rank - 1 if rank > 0 else None, rank + 1 if rank + 1 < world else None)


def exchange(dist, rank, world, send, recv, group=None):
    """Send send[side] to the neighbour on that side and receive recv[side]
    from it, for every side with a neighbour.  send/recv map LOWER/UPPER to
    tensors of equal size; a rank's UPPER message is its upper neighbour's
    LOWER halo and vice versa.  Non-blocking point-to-point, then waits."""
    lo, hi = neighbours(rank, world)
    ops = []
    for side, peer in ((LOWER, lo), (UPPER, hi)):
        if peer is None:
            continue
        ops.append(dist.P2POp(dist.irecv, recv[side], peer, group))
        ops.append(dist.P2POp(dist.isend, send[side], peer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def total(dist, mass, solute, solid_frac, cells, device="cpu", group=None):
    """Whole-grid totals from each rank's own: mass and solute summed, the
    solid fraction weighted by the cells, one FP64 all-reduce."""
    import torch

    v = torch.tensor([mass, float(solid_frac) * cells, float(cells)] + [float(s) for s in solute],
                     dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(v, group=group)
    v = v.cpu().numpy()
    return float(v[0]), np.array(v[3:]), float(v[1] / v[2])


class Slab:
    """One rank's slab: the library handle and its halo messages on the
    device.  step() exchanges and steps once; `transport` moves the packed
    messages (exchange() between ranks, or a copy between two slabs of one
    process)."""

    def __init__(self, sim, rank, world):
        import torch

        self.sim, self.rank, self.world = sim, rank, world
        n = sim.halo_bytes()
        lo, hi = neighbours(rank, world)
        self.sides = [s for s, p in ((LOWER, lo), (UPPER, hi)) if p is not None]
        self.send = {s: torch.empty(n, dtype=torch.uint8, device="cuda") for s in self.sides}
        self.recv = {s: torch.empty(n, dtype=torch.uint8, device="cuda") for s in self.sides}

    def pack(self):
        for s in self.sides:
            self.sim.halo_pack(s, self.send[s])

    def unpack(self):
        for s in self.sides:
            self.sim.halo_unpack(s, self.recv[s])


def step_all(slabs, dist=None):
    """One step of every slab of this process.  With dist (one slab per
    rank) the messages go through exchange(); without it the slabs are
    neighbours in the list order and the messages are copied on the device."""
    for sl in slabs:
        sl.pack()
    if dist is not None:
        for sl in slabs:
            exchange(dist, sl.rank, sl.world, sl.send, sl.recv)
    else:
        for a, b in zip(slabs[:-1], slabs[1:]):
            b.recv[LOWER].copy_(a.send[UPPER])
            a.recv[UPPER].copy_(b.send[LOWER])
    for sl in slabs:
        sl.unpack()
        sl.sim.step(1)
