"""One grid split along y between ranks (slab decomposition), one GPU each.

Rank r of N owns the global rows [r * ny_local, (r + 1) * ny_local) and keeps
two ghost rows on each side (``lbm.Slab``).  Every step is: the local step of
the own rows, then the halo exchange: the two lowest own rows go to rank
r - 1 (its upper ghost rows), the two highest to rank r + 1 (its lower ghost
rows), wrapping around, so the grid stays periodic in y.  The exchange is the
only communication; it moves 2 * 9 * nx elements each way per step.

``exchange`` is independent of what holds the rows: it takes the two packed
halos a rank sends and returns the two it receives, over torch.distributed
point-to-point operations (NCCL for device tensors, gloo for host tensors),
or by a plain swap when one rank holds the whole grid.
"""
from __future__ import annotations


def neighbours(rank: int, world: int):
    """(lower, upper) neighbour ranks, wrapping around."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(low, high, rank: int, world: int, group=None):
    """Sends `low` (the two lowest own rows) to the lower neighbour and `high`
    (the two highest) to the upper one; returns (from_lower, from_upper): the
    lower neighbour's highest rows and the upper neighbour's lowest rows,
    which fill this rank's lower and upper ghost rows.  One rank: its own
    rows wrap around (the periodic grid)."""
    if world == 1:
        return high, low
    import torch
    import torch.distributed as dist
    lower, upper = neighbours(rank, world)
    from_lower = torch.empty_like(high)
    from_upper = torch.empty_like(low)
    # With two ranks the lower and the upper neighbour are the same rank, and
    # messages between a pair match in the order they are posted: the high
    # rows go first, to meet the peer's first receive (its lower ghosts).
    ops = [dist.P2POp(dist.isend, high, upper, group), dist.P2POp(dist.isend, low, lower, group),
           dist.P2POp(dist.irecv, from_lower, lower, group),
           dist.P2POp(dist.irecv, from_upper, upper, group)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return from_lower, from_upper


class SlabRunner:
    """Steps one rank's slab and exchanges its halos.  `slab` provides
    ``step()``, ``pack(side) -> buffer`` and ``unpack(side, buffer)``;
    `swap(low, high) -> (from_lower, from_upper)` is the exchange (for
    example ``functools.partial(exchange, rank=r, world=n)``)."""

    def __init__(self, slab, swap):
        self.slab = slab
        self.swap = swap

    def refresh(self):
        """Fills the ghost rows from the neighbours' current own rows."""
        low, high = self.slab.pack(0), self.slab.pack(1)
        from_lower, from_upper = self.swap(low, high)
        self.slab.unpack(0, from_lower)
        self.slab.unpack(1, from_upper)

    def run(self, steps: int):
        """`steps` time steps of Eq. 5 on the whole split grid (the ghost rows
        are refreshed before the first step and after every step)."""
        self.refresh()
        for _ in range(steps):
            self.slab.step()
            self.refresh()


def run_local(slabs, steps: int):
    """All ranks' slabs in one process (for example several slabs on one
    GPU): the same steps and exchanges as SlabRunner on every rank, the
    exchange done by handing each slab its neighbours' packed rows."""
    world = len(slabs)

    def refresh():
        packs = [(s_.pack(0), s_.pack(1)) for s_ in slabs]
        for r, s_ in enumerate(slabs):
            lower, upper = neighbours(r, world)
            s_.unpack(0, packs[lower][1])
            s_.unpack(1, packs[upper][0])

    refresh()
    for _ in range(steps):
        for s_ in slabs:
            s_.step()
        refresh()


class DeviceSlab:
    """An ``lbm.Slab`` with device halo buffers, in the form SlabRunner and
    run_local take.  The slab's stream must be the current torch stream, so
    that packs, transfers (NCCL runs after the current stream's work and
    makes it wait for the received data) and unpacks are ordered on it."""

    def __init__(self, slab):
        self.grid = slab

    def step(self):
        self.grid.step(1)

    def pack(self, side):
        import torch
        out = torch.empty(self.grid.halo_bytes, dtype=torch.uint8, device="cuda")
        self.grid.pack(side, out)
        return out

    def unpack(self, side, buf):
        self.grid.unpack(side, buf)
