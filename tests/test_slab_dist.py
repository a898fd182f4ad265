"""Slab decomposition in y, on the CPU: ranks of gloo processes each hold
their slab of the grid with two ghost rows on each side, step it with the
FP64 oracle, and exchange the halo rows through the library's exchange
(torch.distributed point-to-point).  The own rows after the run equal the
whole grid's oracle run bit for bit: a step at a row reads values at most two
rows away (the streaming of Eq. 5 and the central gradient of Section 4), so
two ghost rows, refreshed after every step, reproduce the periodic grid
exactly.  The same choreography drives the CUDA slabs (GPU tests)."""
import functools
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from oracle import oracle
from paper_0707_2437_gb300 import slab, workloads

NX, NY_LOCAL, TAU, C2, STEPS = 24, 6, 0.7, 0.21, 25


def _fields(world):
    return workloads.fourier_modes(NX, NY_LOCAL * world, amp=2e-2, seed=world)


class _OracleSlab:
    """Rank r's slab: the oracle state f[9][ny_local + 4][nx] of global rows
    r*ny_local - 2 .. (r+1)*ny_local + 1 (wrapped)."""

    def __init__(self, rank, world):
        rho, ux, uy = _fields(world)
        ny = NY_LOCAL * world
        rows = [(rank * NY_LOCAL - 2 + k) % ny for k in range(NY_LOCAL + 4)]
        self.f = oracle.init(rho[rows], ux[rows], uy[rows])
        self.alpha = oracle.alpha_from_c2(C2)

    def step(self):
        # The periodic oracle on the local buffer: the ghost rows' own
        # results are wrong (they wrap), the own rows' are right.
        oracle.run(self.f, TAU, self.alpha, 1)

    def pack(self, side):
        import torch
        r0 = 2 if side == 0 else NY_LOCAL
        return torch.from_numpy(np.ascontiguousarray(self.f[:, r0:r0 + 2, :]))

    def unpack(self, side, buf):
        r0 = 0 if side == 0 else NY_LOCAL + 2
        self.f[:, r0:r0 + 2, :] = buf.numpy()

    def own(self):
        return self.f[:, 2:NY_LOCAL + 2, :]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.set_threads(1)
        s = _OracleSlab(rank, world)
        runner = slab.SlabRunner(s, functools.partial(slab.exchange, rank=rank, world=world))
        runner.run(STEPS)
        q.put((rank, s.own().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_over_gloo_equal_the_whole_grid(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([parts[r] for r in range(world)], axis=1)
    ref = oracle.init(*_fields(world))
    oracle.run(ref, TAU, oracle.alpha_from_c2(C2), STEPS)
    assert np.array_equal(got, ref)


def test_one_slab_exchanging_with_itself_is_the_periodic_grid():
    s = _OracleSlab(0, 1)
    slab.SlabRunner(s, functools.partial(slab.exchange, rank=0, world=1)).run(STEPS)
    ref = oracle.init(*_fields(1))
    oracle.run(ref, TAU, oracle.alpha_from_c2(C2), STEPS)
    assert np.array_equal(s.own(), ref)


def test_local_run_of_three_slabs_equals_the_whole_grid():
    slabs = [_OracleSlab(r, 3) for r in range(3)]
    slab.run_local(slabs, STEPS)
    got = np.concatenate([s.own() for s in slabs], axis=1)
    ref = oracle.init(*_fields(3))
    oracle.run(ref, TAU, oracle.alpha_from_c2(C2), STEPS)
    assert np.array_equal(got, ref)


def test_neighbours_wrap():
    assert slab.neighbours(0, 4) == (3, 1)
    assert slab.neighbours(3, 4) == (2, 0)
    assert slab.neighbours(0, 1) == (0, 0)
