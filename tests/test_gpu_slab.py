"""Slab decomposition in y on the GPU, all slabs on one device (the exchange
is the same choreography the ranks run over NCCL; here each slab is handed
its neighbours' packed rows): the own rows equal the whole grid's run bit for
bit, and one slab exchanging with itself is the periodic grid."""
import functools

import numpy as np
import pytest

from oracle import oracle
from paper_0707_2437_gb300 import slab, workloads

pytestmark = pytest.mark.gpu


def _local_fields(fields, rank, ny_local):
    ny = fields[0].shape[0]
    rows = [(rank * ny_local - 2 + k) % ny for k in range(ny_local + 4)]
    return [f[rows] for f in fields]


def _slabs(lbm, fields, world, ny_local, tau, c2, storage):
    import torch
    st = torch.cuda.current_stream()
    out = []
    for r in range(world):
        s = lbm.Slab(fields[0].shape[1], ny_local, tau, c2, storage, stream=st)
        s.init(*_local_fields(fields, r, ny_local))
        out.append(slab.DeviceSlab(s))
    return out


@pytest.mark.parametrize("storage", ["f32", "f16d"])
@pytest.mark.parametrize("world,ny_local,nx", [(2, 40, 256), (3, 17, 136), (2, 2, 64)])
def test_slabs_on_one_gpu_equal_the_whole_grid(lbm, storage, world, ny_local, nx):
    tau, c2, steps = 0.7, 0.2, 30
    fields = workloads.fourier_modes(nx, world * ny_local, amp=1e-2, seed=world + nx)
    slabs = _slabs(lbm, fields, world, ny_local, tau, c2, storage)
    slab.run_local(slabs, steps)
    moms = [s.grid.moments() for s in slabs]
    got = [np.concatenate([m[k][2:ny_local + 2] for m in moms]) for k in range(3)]
    with lbm.Grid(nx, world * ny_local, tau, c2, storage) as g:
        g.init(*fields)
        g.step(steps)
        want = g.moments()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    for s in slabs:
        assert s.grid.t == steps
        s.grid.close()


def test_one_slab_with_itself_is_the_periodic_grid_and_matches_oracle(lbm):
    nx, ny, tau, c2, steps = 192, 48, 0.8, 0.3, 50
    fields = workloads.fourier_modes(nx, ny, amp=1e-3, seed=5)
    (s,) = _slabs(lbm, fields, 1, ny, tau, c2, "f32")
    slab.SlabRunner(s, functools.partial(slab.exchange, rank=0, world=1)).run(steps)
    got = [m[2:ny + 2] for m in s.grid.moments()]
    s.grid.close()
    with lbm.Grid(nx, ny, tau, c2) as g:
        g.init(*fields)
        g.step(steps)
        want = g.moments()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    ref = oracle.simulate(*fields, tau, c2, steps)
    assert max(np.abs(a - b).max() for a, b in zip(got, ref)) <= 1e-6


def test_slab_argument_checks(lbm):
    import ctypes
    lib = lbm.load()
    h = ctypes.c_void_p()
    assert lib.lbm_slab_create(64, 1, 0.8, 0.2, 0, None, ctypes.byref(h)) == lbm.LBM_EINVAL
    s = lbm.Slab(64, 8, 0.8, 0.2)
    assert s.ny == 12 and s.halo_bytes == 9 * 2 * 64 * 4
    s.init(*workloads.sine_wave(64, 12))
    assert lib.lbm_step(s.h, 2) == lbm.LBM_EINVAL
    assert lib.lbm_set_drive(s.h, 1, 1e-3, 500.0) == lbm.LBM_EINVAL
    assert lib.lbm_slab_pack(s.h, None, 0) == lbm.LBM_EINVAL
    assert lib.lbm_slab_pack(s.h, ctypes.c_void_p(16), 2) == lbm.LBM_EINVAL
    s.close()
    with lbm.Grid(64, 8, 0.8, 0.2) as g:
        assert lib.lbm_slab_halo_bytes(g.h) == 0
        assert lib.lbm_slab_pack(g.h, ctypes.c_void_p(16), 0) == lbm.LBM_EINVAL
