"""The seeded input recipes (CPU): every workload the tests and the bench use
is drawn as stated, and drawing it twice gives the same numbers, so a change
to a generator cannot silently change a measured workload."""
import numpy as np
import pytest

from paper_0707_2437_gb300 import workloads


def test_sweep_2048_recipe():
    runs = workloads.sweep_2048()
    assert len(runs) == 9
    assert all(r.nx == r.ny == 2048 for r in runs)
    np.testing.assert_allclose([r.c2 for r in runs], 0.05 * np.arange(1, 10), rtol=1e-12)
    assert all(0.55 <= r.tau <= 1.5 for r in runs)
    np.testing.assert_allclose([r.amp for r in runs], np.geomspace(1e-3, 5e-2, 9), rtol=1e-12)
    assert [r.tau for r in runs] == [r.tau for r in workloads.sweep_2048()]


def test_acoustic_shear_fields():
    nx, ny, amp = 64, 5, 2e-3
    rho, ux, uy = workloads.acoustic_shear(nx, ny, amp)
    x = np.arange(nx)
    np.testing.assert_allclose(rho, np.broadcast_to(1 + amp * np.sin(2 * np.pi * x / nx),
                                                    (ny, nx)), rtol=0, atol=1e-16)
    assert not ux.any()
    np.testing.assert_allclose(uy, np.broadcast_to(1e-3 * np.sin(2 * np.pi * x / nx), (ny, nx)),
                               rtol=0, atol=1e-18)


def test_fourier_modes_recipe():
    nx, ny, amp = 96, 40, 1e-3
    rho, ux, uy = workloads.fourier_modes(nx, ny, amp=amp, seed=3)
    assert not ux.any() and not uy.any()
    d = rho - 1.0
    assert abs(np.abs(d).max() - amp) < 1e-18
    # Exactly 8 plane waves with integer wave numbers in [-4, 4]^2 without
    # (0, 0): 8 pairs (k, -k) of nonzero coefficients in the 2-D spectrum.
    spec = np.fft.fft2(d) / (nx * ny)
    big = np.abs(spec) > 1e-9 * amp
    ky, kx = np.nonzero(big)
    kx = np.where(kx > nx // 2, kx - nx, kx)
    ky = np.where(ky > ny // 2, ky - ny, ky)
    assert np.all(np.abs(kx) <= 4) and np.all(np.abs(ky) <= 4)
    assert not np.any((kx == 0) & (ky == 0))
    assert 8 <= big.sum() <= 16  # a pair (k, -k) per wave; two waves may share a pair
    assert np.array_equal(rho, workloads.fourier_modes(nx, ny, amp=amp, seed=3)[0])


def test_batch_grids_recipe():
    runs = workloads.batch_grids()
    assert len(runs) == 512
    nx = np.array([r.nx for r in runs])
    ny = np.array([r.ny for r in runs])
    assert np.all(nx % 8 == 0) and np.all(ny % 8 == 0)
    assert np.all(nx >= 8) and np.all(ny >= 8)
    sites = nx * ny
    # Log-uniform in [64^2, 1024^2] before the sides are rounded to multiples of 8.
    assert sites.min() >= 0.5 * 64 * 64 and sites.max() <= 1.5 * 1024 * 1024
    assert 85e6 < sites.sum() < 105e6
    aspect = nx / ny
    assert aspect.min() >= 0.2 and aspect.max() <= 5.0
    assert all(0.55 <= r.tau <= 1.2 and 0.05 <= r.c2 <= 0.4 for r in runs)
    assert {r.mode for r in runs} == {1, 2, 3}
    assert [(r.nx, r.ny) for r in runs] == [(r.nx, r.ny) for r in workloads.batch_grids()]


def test_serve_trace_recipe():
    reqs = workloads.serve_trace(count=2000, rate_hz=200.0)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) * 200.0 - 1) < 0.05  # Poisson at 200 per second
    assert all(1000 <= r.steps <= 20000 for r in reqs)
    assert all(r.nx % 8 == 0 and r.ny % 8 == 0 for r in reqs)
    sites = np.array([r.nx * r.ny for r in reqs])
    assert sites.min() >= 0.5 * 128 * 128 and sites.max() <= 1.5 * 2048 * 2048
    frac32 = np.mean([r.storage == "f32" for r in reqs])
    assert abs(frac32 - 0.5) < 0.05
    assert {r.storage for r in reqs} == {"f32", "f16d"}
    assert [r.steps for r in reqs] == [r.steps for r in workloads.serve_trace(count=2000,
                                                                              rate_hz=200.0)]


@pytest.mark.parametrize("u0,c", [(2e-3, 0.2), (2e-3, 0.9)])
def test_progressive_wave_reading(u0, c):
    """Section 4's progressive wave, read as rho = rho0 (1 + (u0/c) sin kx),
    u_x = u0 sin kx."""
    nx, ny = 128, 4
    rho, ux, uy = workloads.progressive_wave(nx, ny, u0, c)
    s = np.sin(2 * np.pi * np.arange(nx) / nx)
    np.testing.assert_allclose(rho[0], 1 + (u0 / c) * s, rtol=0, atol=1e-16)
    np.testing.assert_allclose(ux[0], u0 * s, rtol=0, atol=1e-18)
    assert not uy.any()


def test_c2_lens_recipe():
    nx, ny, c2 = 200, 120, 0.2
    f = workloads.c2_lens(nx, ny, c2, contrast=0.5, width=0.15)
    assert f.shape == (ny, nx)
    assert abs(f.max() / c2 - 1.5) < 0.01      # raised by half at the centre
    assert abs(f.min() / c2 - 1.0) < 0.01      # ambient far from it
    assert np.unravel_index(np.argmax(f), f.shape) in [(ny // 2 - 1, nx // 2 - 1),
                                                        (ny // 2 - 1, nx // 2),
                                                        (ny // 2, nx // 2 - 1),
                                                        (ny // 2, nx // 2)]
