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


def _solo(lbm, nx, ny, tau, c2, storage, field, fields, steps, rounding=None, persistent=True):
    with lbm.Grid(nx, ny, tau, c2, storage) as g:
        g.set_persistent(persistent)
        if rounding:
            g.set_rounding(rounding)
        if field is not None:
            g.set_c2_field(field)
        g.init(*fields)
        g.step(steps)
        return g.get_state()[0]


@pytest.mark.parametrize("storage", ["f32", "f16d", "bf16d"])
def test_persistent_steps_with_field_equal_step_kernel(lbm, storage):
    """Long lbm_step calls run the persistent batch kernel also with a c2
    field; the state equals the step kernel's bit for bit."""
    nx, ny = 256, 96
    f = workloads.fourier_modes(nx, ny, amp=1e-3, seed=4)
    c2 = _c2_field(nx, ny)
    a = _solo(lbm, nx, ny, 0.7, 0.2, storage, c2, f, 150, persistent=True)
    b = _solo(lbm, nx, ny, 0.7, 0.2, storage, c2, f, 150, persistent=False)
    assert np.array_equal(a, b)


def test_field_grids_in_batch_equal_solo_runs(lbm):
    """Grids with and without c2 fields, FP32 and 16-bit, some with nx not a
    multiple of 4 and one large enough for its own launch, stepped together
    with per-grid limits: each reaches bitwise its solo state."""
    specs = [(2048, 512, "f32", True), (256, 40, "f16d", True), (37, 23, "f32", True),
             (128, 64, "bf16d", False), (96, 30, "f32", False), (130, 9, "bf16d", True)]
    limits = [20, 33, 40, 12, 40, 7]
    fields, solo = [], []
    for (nx, ny, st, fld), lim in zip(specs, limits):
        f = workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny)
        c2 = _c2_field(nx, ny) if fld else None
        fields.append((f, c2))
        solo.append(_solo(lbm, nx, ny, 0.75, 0.2, st, c2, f, lim))
    grids = []
    for (nx, ny, st, fld), (f, c2) in zip(specs, fields):
        g = lbm.Grid(nx, ny, 0.75, 0.2, st)
        if c2 is not None:
            g.set_c2_field(c2)
        g.init(*f)
        grids.append(g)
    b = lbm.Batch(grids)
    assert b.get_config()["groups"] >= 2
    b.step(25, limits)
    b.step(15, [max(0, x - 25) for x in limits])
    assert b.sync() == 0
    for g, s_, lim in zip(grids, solo, limits):
        assert g.t == lim
        assert np.array_equal(g.get_state()[0], s_)
    b.close()
    for g in grids:
        g.close()


def test_batch_follows_field_and_rounding_set_after_creation(lbm):
    """A c2 field or stochastic rounding set on a grid after its batch was
    built takes effect at the next step call (the work-list is rebuilt)."""
    nx, ny = 192, 48
    f = workloads.fourier_modes(nx, ny, amp=1e-3, seed=9)
    c2 = _c2_field(nx, ny)
    want_field = _solo(lbm, nx, ny, 0.8, 0.25, "f32", c2, f, 30)
    want_sr = _solo(lbm, nx, ny, 0.8, 0.25, "f16d", None, f, 30, rounding="stochastic")
    a = lbm.Grid(nx, ny, 0.8, 0.25, "f32")
    h = lbm.Grid(nx, ny, 0.8, 0.25, "f16d")
    a.init(*f)
    h.init(*f)
    b = lbm.Batch([a, h])
    a.set_c2_field(c2)
    h.set_rounding("stochastic")
    b.step(30)
    assert b.sync() == 0
    assert np.array_equal(a.get_state()[0], want_field)
    assert np.array_equal(h.get_state()[0], want_sr)
    b.close()
    a.close()
    h.close()
