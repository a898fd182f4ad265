"""Grids at the size limit (nx * ny just below 2^31 sites): the nine planes
span about 1.9e10 element offsets, so any 32-bit index arithmetic would show
here.  A y-uniform plane wave must evolve identically in every row, so the
grid's FP64 Fourier mode and totals equal those of a 4-row grid of the same
width stepped the same way."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _plane_wave_on_device(torch, nx, ny, amp):
    x = torch.arange(nx, dtype=torch.float64, device="cuda")
    row = 1.0 + amp * torch.sin(2 * np.pi * x / nx)
    rho = row.expand(ny, nx).contiguous()
    z = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    uy = z.clone()
    return rho, z, uy


@pytest.mark.parametrize("storage,nx,ny", [("f16d", 65536, 32767), ("f32", 65536, 16384)])
def test_grid_at_size_limit_evolves_every_row_alike(lbm, storage, nx, ny):
    torch = pytest.importorskip("torch")
    need = lbm.bytes_required(nx, ny, storage) + 3 * 8 * nx * ny
    free, _ = lbm.mem_info()
    if need > 0.8 * free:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    amp, tau, c2 = 1e-3, 0.7, 0.2
    results = []
    for rows in (ny, 4):
        with lbm.Grid(nx, rows, tau, c2, storage) as g:
            fields = _plane_wave_on_device(torch, nx, rows, amp)
            g.init(*fields)
            del fields
            torch.cuda.empty_cache()
            g.step(3)    # step-kernel launches
            g.step(40)   # one persistent launch
            m1 = g.mode("rho", 1, 0)
            mxy = g.mode("rho", 1, 1)
            sums = g.sums() / (nx * rows)
            results.append((m1, mxy, sums))
    (m_big, mxy_big, s_big), (m_small, _, s_small) = results
    print(f"{storage} {nx}x{ny}: mode {m_big}, 4-row grid {m_small}")
    assert np.abs(m_big - m_small).max() <= 1e-9 * amp
    assert np.abs(mxy_big).max() <= 1e-9 * amp      # no y structure anywhere
    assert np.abs(s_big - s_small).max() <= 1e-12
    assert 0.5 * amp < np.hypot(*m_big) < 1.01 * amp  # the wave is still there
