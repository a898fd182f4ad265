"""lbm_sums_noalloc: the grid totals for callers that cannot allocate device
memory (their own memory pools, up-front memory budgets, or places where no
allocating CUDA call may be made).  Its reduction scratch is a fixed array in
the library's device memory instead of a buffer owned by a handle.

The test checks it against lbm_sums, through the C ABI, on two calls in a row
(different grids and storages, so the second call reuses the scratch the first
one left behind).  This file is collected last so that a stop at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_0707_2437_gb300 import workloads

pytestmark = pytest.mark.gpu


def _state_on_device(g):
    """The grid's state copied to a fresh device buffer in the checkpoint
    layout (9 planes of nx*ny elements)."""
    import torch
    raw, _ = g.get_state()
    return torch.from_numpy(raw).cuda()


def test_sums_noalloc_matches_lbm_sums_twice(lbm):
    import torch
    cases = [(192, 80, 0.7, 0.2, "f32", 40), (256, 37, 0.9, 0.1, "f16d", 25)]
    for nx, ny, tau, c2, storage, steps in cases:
        rho, ux, uy = workloads.fourier_modes(nx, ny, amp=1e-2, seed=nx)
        ux = ux + 1e-3 * np.cos(2 * np.pi * np.arange(ny) / ny)[:, None]
        with lbm.Grid(nx, ny, tau, c2, storage) as g:
            g.init(rho, ux, uy)
            g.step(steps)
            want = g.sums()
            dev = _state_on_device(g)
            torch.cuda.synchronize()
            got = lbm.sums_noalloc(dev.data_ptr(), nx, ny, nx * ny, storage)
        # Same reduction order as lbm_sums: equal to FP64 rounding.
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * nx * ny)


def test_sums_noalloc_padded_planes_bf16_and_own_stream(lbm):
    """The other inputs the header documents: BF16-delta storage, planes
    padded apart (plane_stride > nx*ny, so plane i starts at i*plane_stride),
    and a caller's non-default stream; again two calls in a row."""
    import torch
    pad = 37
    stream = torch.cuda.Stream()
    for nx, ny, storage, steps in [(160, 41, "bf16d", 30), (96, 50, "f32", 12)]:
        rho, ux, uy = workloads.fourier_modes(nx, ny, amp=2e-2, seed=nx + 1)
        uy = uy + 2e-3 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :]
        with lbm.Grid(nx, ny, 0.75, 0.15, storage) as g:
            g.init(rho, ux, uy)
            g.step(steps)
            want = g.sums()
            raw, _ = g.get_state()
        n = nx * ny
        esize = 4 if storage == "f32" else 2
        planes = torch.from_numpy(raw.view(np.uint8)).view(9, n * esize)
        padded = torch.full((9, (n + pad) * esize), 0xFF, dtype=torch.uint8)
        padded[:, :n * esize] = planes  # the gaps hold NaN patterns: never read
        dev = padded.cuda()
        torch.cuda.synchronize()
        got = lbm.sums_noalloc(dev.data_ptr(), nx, ny, n + pad, storage, stream=stream)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * n)


def test_sums_noalloc_rejects_bad_sizes(lbm):
    lib = lbm.load()
    out = (np.zeros(3))
    import ctypes
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.lbm_sums_noalloc(ctypes.c_void_p(16), 70000, 70000, 70000 * 70000, 0, 1.0,
                                None, p) == -1
    assert lib.lbm_sums_noalloc(ctypes.c_void_p(16), 8, 8, 63, 0, 1.0, None, p) == -1
