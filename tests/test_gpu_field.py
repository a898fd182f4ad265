"""Spatially varying sound speed: a per-site c^2 (alpha = 1/3 - c^2 at each
site in the force of Section 3, Eq. 5; the paper's Section 5 outlook)."""
import numpy as np
import pytest

from oracle import oracle
from paper_0707_2437_gb300 import workloads

pytestmark = pytest.mark.gpu


def _c2_field(nx, ny):
    x = np.arange(nx)[None, :] / nx
    y = np.arange(ny)[:, None] / ny
    return 0.2 + 0.12 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-6), ("f16d", 2e-5), ("bf16d", 2e-4)])
@pytest.mark.parametrize("nx,ny", [(256, 48), (37, 23), (130, 9)])
def test_c2_field_matches_oracle(lbm, storage, tol, nx, ny):
    """GPU with a c^2 field against the oracle with the same per-site alpha."""
    rho, ux, uy = workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx)
    c2 = _c2_field(nx, ny)
    tau, steps = 0.7, 150
    with lbm.Grid(nx, ny, tau, 0.2, storage) as g:
        g.set_c2_field(c2)
        g.init(rho, ux, uy)
        g.step(steps)
        got = g.moments()
    f = oracle.init(rho, ux, uy)
    oracle.run(f, tau, 1.0 / 3.0 - c2, steps)
    ref = oracle.moments(f)
    err = max(np.abs(a - b).max() for a, b in zip(got, ref))
    assert err <= tol, err


def test_uniform_field_equals_uniform_c2_bitwise(lbm):
    nx, ny, c2 = 200, 30, 0.15
    f = workloads.fourier_modes(nx, ny, amp=1e-3, seed=1)
    out = []
    for field in (None, np.full((ny, nx), c2)):
        with lbm.Grid(nx, ny, 0.8, c2) as g:
            g.set_persistent(False)
            if field is not None:
                g.set_c2_field(field)
            g.init(*f)
            g.step(40)
            out.append(g.get_state()[0])
    assert np.array_equal(out[0], out[1])


def test_pulse_travel_time_follows_local_sound_speed(lbm):
    """A density pulse crossing a smooth step from c^2 = 0.1 to 0.4 reaches a
    probe at the time integral of dx / c(x) (ray travel time)."""
    nx, ny, tau = 4096, 4, 0.55
    x = np.arange(nx, dtype=float)
    c2x = 0.1 + 0.3 * 0.5 * (1 + np.tanh((x - 2048) / 40.0))
    c2 = np.broadcast_to(c2x, (ny, nx)).copy()
    x0, x1 = 1024, 3072
    rho = np.broadcast_to(1 + 1e-4 * np.exp(-0.5 * ((x - x0) / 6.0) ** 2), (ny, nx)).copy()
    z = np.zeros((ny, nx))
    t_theory = float(np.sum(1.0 / np.sqrt(c2x[x0:x1])))
    with lbm.Grid(nx, ny, tau, 0.25) as g:
        g.set_c2_field(c2)
        g.init(rho, z, z.copy())
        t_lo = int(0.9 * t_theory)
        g.step(t_lo)
        ts, vals = [], []
        while g.t < 1.1 * t_theory:
            r, _, _ = g.moments()
            ts.append(g.t)
            vals.append(r[:, x1].mean() - 1.0)
            g.step(4)
    t_peak = ts[int(np.argmax(vals))]
    print(f"pulse arrival {t_peak} steps, ray time {t_theory:.0f}")
    assert abs(t_peak / t_theory - 1) < 0.02


def test_batch_rejects_field_grids(lbm):
    g = lbm.Grid(64, 8, 0.8, 0.2)
    g.set_c2_field(np.full((8, 64), 0.3))
    with pytest.raises(lbm.LbmError):
        lbm.Batch([g])
    g.close()
