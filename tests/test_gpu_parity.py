"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances.  The FP32 path stores h_i = (f_i - w_i)/w_i and does FP32
arithmetic on quantities of the size of the density deviation A, so a step
adds rounding of about 2^-24 A per site; after n steps the error stays well
below n * 2^-24 * A * (a few).  The bar is the stated one: max |rho - rho_ref|
<= 1e-6 after 1000 steps at amplitude 1e-3 (64 x 64), applied to every case
below.  The 16-bit storages round h_i on every store (FP16: 2^-11 relative,
BF16: 2^-8 relative); their bounds are stated in test_sixteen_bit_storage.
"""
import numpy as np
import pytest

from oracle import linear, oracle
from paper_0707_2437_gb300 import workloads
from tests.helpers import fit_damped_cos, fit_decay

pytestmark = pytest.mark.gpu

F32_TOL = 1e-6


def _fields(nx, ny, amp=1e-3, seed=0, u=1e-4):
    rho, ux, uy = workloads.fourier_modes(nx, ny, amp=amp, seed=seed)
    rng = np.random.default_rng(seed + 100)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    ux = u * np.sin(2 * np.pi * y / ny + rng.uniform(0, 6)) * np.ones((1, nx))
    uy = u * np.cos(2 * np.pi * x / nx + rng.uniform(0, 6)) * np.ones((ny, 1))
    return rho, ux, uy


def _run_gpu(lbm, nx, ny, tau, c2, fields, steps, storage="f32", cfg=None):
    with lbm.Grid(nx, ny, tau, c2, storage) as g:
        if cfg:
            g.set_config(*cfg)
        g.init(*fields)
        g.step(steps)
        return g.moments()


def _err(a, b):
    return max(np.abs(x - y).max() for x, y in zip(a, b))


@pytest.mark.parametrize("c2", [1 / 3, 0.2])
def test_config_64x64_1000_steps(lbm, c2):
    """The 64 x 64 case: rho = 1 + 1e-3 sin(2 pi x/64), u = 0, tau = 0.8,
    1000 steps: max |rho - rho_ref| <= 1e-6 (FP32)."""
    f = workloads.sine_wave(64, 64, 1e-3)
    got = _run_gpu(lbm, 64, 64, 0.8, c2, f, 1000)
    ref = oracle.simulate(*f, 0.8, c2, 1000)
    assert np.abs(got[0] - ref[0]).max() <= F32_TOL
    assert _err(got, ref) <= F32_TOL


@pytest.mark.parametrize("nx,ny", [(200, 50), (37, 23), (130, 7), (256, 9), (8, 3), (3, 3),
                                   (1, 5), (5, 1), (2, 2), (384, 33)])
def test_fp32_matches_oracle_many_shapes(lbm, nx, ny):
    """Odd sizes, ragged tails, strips narrower than a warp, several strips
    per row and the degenerate 1- and 2-site periods (central difference of
    zero along that axis)."""
    rng = np.random.default_rng(nx * 1000 + ny)
    tau = float(rng.uniform(0.55, 1.5))
    c2 = float(rng.uniform(0.05, 0.6))
    f = _fields(nx, ny, seed=nx + ny)
    got = _run_gpu(lbm, nx, ny, tau, c2, f, 120)
    ref = oracle.simulate(*f, tau, c2, 120)
    assert _err(got, ref) <= F32_TOL


def test_every_tile_configuration_bitwise_identical(lbm):
    """The step's result does not depend on the tile shape, lanes per site or
    block size (the same FP32 operations in the same order everywhere)."""
    nx, ny = 256, 45
    f = _fields(nx, ny, seed=5)
    states = {}
    for vec in (1, 2, 4):
        for rows in (1, 3, 16, 64):
            for warps in (1, 4, 8):
                for stages in {4: (0, 2, 3, 4), 2: (0, 1)}.get(vec, (0,)):
                    with lbm.Grid(nx, ny, 0.7, 0.15, "f32") as g:
                        g.set_config(vec, rows, warps)
                        g.set_pipeline(stages)
                        assert g.get_pipeline() == (stages, stages > 0)
                        g.init(*f)
                        g.step(13)
                        states[(vec, rows, warps, stages)] = g.get_state()[0]
    ref = states[(4, 16, 4, 0)]
    for k, s in states.items():
        assert np.array_equal(s, ref), k


@pytest.mark.parametrize("storage", ["f16d", "bf16d"])
def test_sixteen_bit_tile_configurations_bitwise(lbm, storage):
    nx, ny = 512, 20
    f = _fields(nx, ny, seed=6)
    states = []
    for vec, rows, warps, stages in ((8, 16, 4, 0), (8, 16, 4, 4), (8, 5, 8, 2), (8, 33, 1, 3),
                                     (4, 7, 2, 0), (4, 7, 2, 1), (4, 16, 8, 1), (8, 9, 8, 1), (8, 3, 2, 1),
                                     (2, 5, 8, 0),
                                     (1, 64, 1, 0)):
        with lbm.Grid(nx, ny, 0.9, 0.3, storage) as g:
            g.set_config(vec, rows, warps)
            g.set_pipeline(stages)
            g.init(*f)
            g.step(11)
            states.append(g.get_state()[0])
    for s in states[1:]:
        assert np.array_equal(s, states[0])


@pytest.mark.parametrize("storage", ["f32", "f16d", "bf16d"])
@pytest.mark.parametrize("nx,ny", [(8, 3), (16, 5), (136, 9), (264, 17), (520, 33), (1032, 6)])
def test_pipeline_strip_edges_match_register_walk(lbm, storage, nx, ny):
    """The bulk-copy pipeline's wrapped row pieces (strips at x = 0, at the
    right edge, strips that are the whole row, partial last strips) give the
    register walk's bits."""
    vec = 4 if storage == "f32" else 8
    if nx % vec:
        pytest.skip("vector width does not divide nx")
    f = _fields(nx, ny, seed=nx + 3)
    out = []
    for stages in (0, 3):
        with lbm.Grid(nx, ny, 0.8, 0.2, storage) as g:
            g.set_config(vec, 4, 2)
            g.set_pipeline(stages)
            g.init(*f)
            g.step(9)
            out.append(g.get_state()[0])
    assert np.array_equal(out[0], out[1])
    if storage == "f32":
        got = _run_gpu(lbm, nx, ny, 0.8, 0.2, f, 9, cfg=(vec, 4, 2))
        assert _err(got, oracle.simulate(*f, 0.8, 0.2, 9)) <= F32_TOL


@pytest.mark.parametrize("storage", ["f16d", "bf16d"])
def test_stochastic_rounding_configs_graphs_and_batch_bitwise(lbm, storage):
    """Stochastic rounding is seeded by (site, direction, step) only: every
    register-walk configuration, graph replay against single launches, and
    the batched kernel give the same bits."""
    nx, ny = 256, 40
    f = _fields(nx, ny, seed=21)
    states = []
    for vec, rows, warps, stages in ((4, 16, 4, 1), (4, 7, 2, 0), (2, 5, 8, 0), (1, 64, 1, 0)):
        with lbm.Grid(nx, ny, 0.7, 0.12, storage) as g:
            g.set_rounding("stochastic")
            g.set_config(vec, rows, warps)
            g.set_pipeline(stages)
            g.init(*f)
            g.step(37)  # one graph of 32 steps plus single launches
            states.append(g.get_state()[0])
    for st in states[1:]:
        assert np.array_equal(st, states[0])
    with lbm.Grid(nx, ny, 0.7, 0.12, storage) as g:
        g.set_rounding("stochastic")
        g.init(*f)
        for _ in range(37):
            g.step(1)
        assert np.array_equal(g.get_state()[0], states[0])
    g = lbm.Grid(nx, ny, 0.7, 0.12, storage)
    g.set_rounding("stochastic")
    g.init(*f)
    other = lbm.Grid(64, 64, 0.8, 0.2, "f32")
    other.init(*_fields(64, 64, seed=3))
    b = lbm.Batch([g, other])
    b.step(37)
    assert b.sync() == 0
    assert np.array_equal(g.get_state()[0], states[0])
    b.close()
    g.close()
    other.close()
    # Nearest and stochastic rounding differ (the setting takes effect).
    with lbm.Grid(nx, ny, 0.7, 0.12, storage) as h:
        h.init(*f)
        h.step(37)
        assert not np.array_equal(h.get_state()[0], states[0])


def test_rounding_mode_validation(lbm):
    with lbm.Grid(64, 8, 0.8, 0.2, "f32") as g:
        with pytest.raises(lbm.LbmError):
            g.set_rounding("stochastic")
    with lbm.Grid(64, 8, 0.8, 0.2, "f16d") as g:
        g.set_config(8, 16, 8)  # 8 warps: no shared-memory walk at this block size
        g.set_rounding("stochastic")
        assert g.get_config()[0] == 4
        assert g.get_rounding() == "stochastic"
        with pytest.raises(lbm.LbmError):
            g.set_config(8, 16, 8)
        g.set_config(8, 16, 4)  # the shared-memory walk takes stochastic rounding
        assert g.get_config()[0] == 8
        with pytest.raises(lbm.LbmError):
            g.set_pipeline(3)


@pytest.mark.parametrize("storage", ["f16d", "bf16d"])
@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
def test_step_kernel_8_site_walk_equals_other_walks(lbm, storage, rounding):
    """The step kernel's 8-site walk with rows through shared memory leaves the
    state bit for bit equal to the 4-site register walk and to the batch
    kernel, with either rounding."""
    nx, ny = 256, 40
    f = _fields(nx, ny, seed=11)
    out = []
    for cfg in ((8, 16, 4), (8, 5, 4), (4, 16, 4), None):
        with lbm.Grid(nx, ny, 0.7, 0.25, storage) as g:
            if rounding != "nearest":
                g.set_rounding(rounding)
            g.init(*f)
            if cfg is None:
                b = lbm.Batch([g])
                b.step(30)
                assert b.sync() == 0
                b.close()
            else:
                g.set_config(*cfg)
                g.set_persistent(False)
                g.step(30)
            out.append(g.get_state()[0])
    for o in out[1:]:
        assert np.array_equal(out[0], o)


@pytest.mark.parametrize("storage,rounding", [("f32", "nearest"), ("f16d", "nearest"),
                                              ("bf16d", "stochastic")])
@pytest.mark.parametrize("nx,ny", [(256, 100), (37, 23), (520, 9)])
def test_persistent_long_steps_equal_step_kernel(lbm, storage, rounding, nx, ny):
    """lbm_step runs long calls as one persistent launch; the state equals the
    step kernel's (persistent mode off) bit for bit."""
    f = _fields(nx, ny, seed=nx + 7)
    out = []
    for persistent in (True, False):
        with lbm.Grid(nx, ny, 0.75, 0.18, storage) as g:
            if rounding != "nearest":
                g.set_rounding(rounding)
            g.set_persistent(persistent)
            g.init(*f)
            g.step(150)
            g.step(3)
            g.step(70)
            assert g.t == 223
            out.append(g.get_state()[0])
    assert np.array_equal(out[0], out[1])


def test_graph_replay_equals_single_launches(lbm):
    nx, ny = 96, 64
    f = _fields(nx, ny, seed=7)
    with lbm.Grid(nx, ny, 0.8, 0.2) as a, lbm.Grid(nx, ny, 0.8, 0.2) as b:
        a.init(*f)
        b.init(*f)
        a.step(77)           # graphs of 32 steps plus single launches
        for _ in range(77):
            b.step(1)
        assert a.t == b.t == 77
        assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_checkpoint_resume_bitwise(lbm):
    nx, ny = 128, 40
    f = _fields(nx, ny, seed=8)
    with lbm.Grid(nx, ny, 0.6, 0.1) as a:
        a.init(*f)
        a.step(50)
        st, t = a.get_state()
        a.step(31)
        end = a.get_state()[0]
    with lbm.Grid(nx, ny, 0.6, 0.1) as b:
        b.set_state(st, t)
        assert b.t == 50
        b.step(31)
        assert b.t == 81
        assert np.array_equal(b.get_state()[0], end)


def test_sums_and_modes_match_oracle(lbm):
    nx, ny, tau, c2, steps = 160, 48, 0.75, 0.25, 60
    f = _fields(nx, ny, seed=9, u=1e-3)
    fo = oracle.init(*f)
    with lbm.Grid(nx, ny, tau, c2) as g:
        g.init(*f)
        s0 = g.sums()
        # FP32 storage of the initial state: N sites x 2^-24 x 1e-3 at most.
        np.testing.assert_allclose(s0, oracle.sums(fo), rtol=0, atol=2e-6)
        g.step(steps)
        oracle.run(fo, tau, oracle.alpha_from_c2(c2), steps)
        s1 = g.sums()
        ref = oracle.sums(fo)
        np.testing.assert_allclose(s1, ref, rtol=0, atol=2e-6)
        r, u, v = oracle.moments(fo)
        x = np.arange(nx)[None, :] / nx
        y = np.arange(ny)[:, None] / ny
        for field, val in (("rho", r - 1.0), ("ux", u), ("uy", v)):
            for kx, ky in ((1, 0), (0, 1), (2, -1), (3, 2)):
                ph = 2 * np.pi * (kx * x + ky * y)
                want = 2.0 / (nx * ny) * np.array([(val * np.cos(ph)).sum(),
                                                   (val * np.sin(ph)).sum()])
                np.testing.assert_allclose(g.mode(field, kx, ky), want, rtol=0, atol=1e-9)


def test_conservation_on_gpu(lbm):
    """Mass and momentum totals (FP64 reductions of the stored state) stay at
    their initial values to FP32 rounding over 500 steps."""
    nx, ny = 512, 256
    f = _fields(nx, ny, amp=1e-2, seed=10, u=1e-3)
    with lbm.Grid(nx, ny, 0.7, 0.12) as g:
        g.init(*f)
        s0 = g.sums()
        g.step(500)
        s1 = g.sums()
    n = nx * ny
    # 500 steps x 2^-24 relative rounding of values of size 1e-2 per site,
    # summed over n sites with random signs: far below 1e-6 n.
    assert abs(s1[0] - s0[0]) < 1e-6 * n * 1e-2
    assert np.all(np.abs(s1[1:] - s0[1:]) < 1e-6 * n * 1e-2)


@pytest.mark.parametrize("c2", [1 / 3, 0.2, 0.05])
def test_gpu_sound_speed_matches_linear_theory(lbm, c2):
    """Standing wave at amplitude 1e-6 on the GPU: the fitted frequency of the
    FP64 mode amplitude equals the linear analysis (Section 3, Eq. 8 at this
    k) to 1e-5 and sqrt(c2) to the grid's O(k^2) offset."""
    nx, tau = 128, 0.8
    k = 2 * np.pi / nx
    alpha = 1 / 3 - c2
    lin = linear.hydro_modes(k, 0, tau, alpha)
    period = 2 * np.pi / lin["omega"]
    every = max(1, int(period / 50))
    f = workloads.sine_wave(nx, 4, 1e-6)
    ts, amps = [], []
    with lbm.Grid(nx, 4, tau, c2) as g:
        g.init(*f)
        while g.t <= 3 * period:
            ts.append(g.t)
            amps.append(g.mode("rho", 1, 0)[1])
            g.step(every)
    ts, amps = np.array(ts, float), np.array(amps)
    keep = ts >= 20
    w, gam, _, _ = fit_damped_cos(ts[keep], amps[keep], lin["omega"], lin["gamma_sound"])
    assert abs(w / lin["omega"] - 1) < 1e-5
    assert abs(w / k / np.sqrt(c2) - 1) < 2e-3


def test_gpu_shear_viscosity_independent_of_c(lbm):
    """Shear-wave decay on the GPU: nu = (2 tau - 1)/6 for every c2."""
    nx, tau = 128, 0.9
    k = 2 * np.pi / nx
    nu = (2 * tau - 1) / 6
    rates = []
    for c2 in (1 / 3, 0.2, 0.05):
        rho = np.ones((4, nx))
        uy = np.broadcast_to(1e-4 * np.sin(k * np.arange(nx)), (4, nx)).copy()
        ts, amps = [], []
        with lbm.Grid(nx, 4, tau, c2) as g:
            g.init(rho, np.zeros((4, nx)), uy)
            for _ in range(20):
                ts.append(g.t)
                amps.append(g.mode("uy", 1, 0)[1])
                g.step(50)
        rates.append(fit_decay(np.array(ts[2:], float), np.array(amps[2:])))
    rates = np.array(rates)
    assert np.all(np.abs(rates / (nu * k * k) - 1) < 2e-3)
    assert np.ptp(rates) / rates.mean() < 1e-5


@pytest.mark.parametrize("storage,tol_rho,tol_u", [("f16d", 2e-5, 2e-5), ("bf16d", 2e-4, 2e-4)])
def test_sixteen_bit_storage(lbm, storage, tol_rho, tol_u):
    """16-bit delta storage against the FP64 oracle, amplitude 1e-3,
    500 steps.  FP16 keeps 11 significant bits of h (about 5e-7 absolute at
    this amplitude per store), BF16 8 bits (about 4e-6): the stated bounds."""
    nx, ny, tau, c2, steps = 256, 64, 0.6, 0.15, 500
    f = workloads.fourier_modes(nx, ny, amp=1e-3, seed=3)
    got = _run_gpu(lbm, nx, ny, tau, c2, f, steps, storage)
    ref = oracle.simulate(*f, tau, c2, steps)
    e_rho = np.abs(got[0] - ref[0]).max()
    e_u = max(np.abs(got[1] - ref[1]).max(), np.abs(got[2] - ref[2]).max())
    print(f"{storage}: max|drho| = {e_rho:.3e}, max|du| = {e_u:.3e}")
    assert e_rho <= tol_rho
    assert e_u <= tol_u


def test_sampled_sites_at_full_2048_size(lbm):
    """2048 x 2048 (the bench's grid and default launch configuration): all
    sites' moments after 10 steps against a 10-step FP64 oracle run of the
    whole grid."""
    n = 2048
    runs = workloads.sweep_2048(n)
    r = runs[4]
    f = workloads.acoustic_shear(n, n, r.amp)
    with lbm.Grid(n, n, r.tau, r.c2) as g:
        g.init(*f)
        g.step(10)
        got = g.moments()
    ref = oracle.simulate(*f, r.tau, r.c2, 10)
    assert _err(got, ref) <= 1e-7


def test_batch_equals_solo_runs(lbm):
    """Grids of different sizes, tau, c2 and storage stepped together in one
    persistent launch give bitwise the state each reaches alone, including
    grids that stop early (per-grid step limits)."""
    specs = [(64, 64, 0.8, 0.2, "f32"), (37, 23, 0.6, 0.1, "f32"), (256, 40, 1.1, 0.3, "f16d"),
             (96, 130, 0.55, 0.05, "bf16d"), (8, 8, 0.9, 0.4, "f32"), (520, 16, 0.7, 0.25, "f32")]
    limits = [40, 40, 25, 40, 3, 40]
    solo = []
    for (nx, ny, tau, c2, st), lim in zip(specs, limits):
        with lbm.Grid(nx, ny, tau, c2, st) as g:
            g.init(*_fields(nx, ny, seed=nx))
            g.step(lim)
            solo.append(g.get_state()[0])
    grids = []
    for nx, ny, tau, c2, st in specs:
        g = lbm.Grid(nx, ny, tau, c2, st)
        g.init(*_fields(nx, ny, seed=nx))
        grids.append(g)
    b = lbm.Batch(grids)
    b.step(30, limits)
    b.step(10, [max(0, x - 30) for x in limits])
    assert b.sync() == 0
    for g, s, lim in zip(grids, solo, limits):
        assert g.t == lim
        assert np.array_equal(g.get_state()[0], s)
    b.close()
    for g in grids:
        g.close()


def test_batch_barrier_timeout_reports_status(lbm):
    """A barrier wait limit of 1 microsecond runs out while other blocks are
    still working: the kernel ends, the host reads LBM_ETIMEOUT, and the
    context stays usable (the next run with a normal limit succeeds)."""
    grids = [lbm.Grid(1024, 1024, 0.8, 0.2) for _ in range(2)]
    for g in grids:
        g.init(*workloads.sine_wave(1024, 1024))
    b = lbm.Batch(grids)
    # 16-row tiles: 1024 of them, one walk of about 30 us each, so blocks
    # without a tile wait at the barrier far longer than the limit.
    b.set_config(16, 0)
    b.set_timeout_us(1)
    b.step(20)
    with pytest.raises(lbm.LbmError) as ei:
        b.sync()
    assert ei.value.status == lbm.LBM_ETIMEOUT
    b.set_timeout_us(1_000_000)
    for g in grids:
        g.init(*workloads.sine_wave(1024, 1024))
    b.step(5)
    assert b.sync() == 0
    assert all(g.t == 5 for g in grids)
    b.close()
    for g in grids:
        g.close()


def test_autotune_keeps_results_and_cache(lbm, tmp_path):
    nx, ny = 512, 128
    f = _fields(nx, ny, seed=11)
    cache = str(tmp_path / "tune.json")
    with lbm.Grid(nx, ny, 0.8, 0.2) as g:
        g.init(*f)
        st0 = g.get_state()[0]
        cfg = g.tune(cache)
        assert np.array_equal(g.get_state()[0], st0)  # tuning does not step
        assert g.t == 0
    with lbm.Grid(nx, ny, 0.8, 0.2) as h:
        assert h.tune(cache) == cfg  # read back from the cache
    import json
    assert len(json.load(open(cache))) == 1


@pytest.mark.parametrize("storage", ["f32", "f16d"])
def test_large_grid_short_calls_persistent_equal_single_launches(lbm, storage):
    """On a grid of 2^20 sites, calls of 8 to 63 steps also run as one
    persistent launch; the state equals single-step launches bit for bit."""
    nx, ny = 1024, 1024
    f = _fields(nx, ny, seed=11)
    with lbm.Grid(nx, ny, 0.7, 0.25, storage) as a, lbm.Grid(nx, ny, 0.7, 0.25, storage) as b:
        a.init(*f)
        b.init(*f)
        a.step(8)
        a.step(13)
        for _ in range(21):
            b.step(1)
        assert a.t == b.t == 21
        assert np.array_equal(a.get_state()[0], b.get_state()[0])


@pytest.mark.parametrize("storage", ["f32", "f16d", "bf16d"])
def test_y_uniform_state_stays_y_uniform_on_gpu(lbm, storage):
    """A y-uniform plane wave stays exactly y-uniform on the GPU (every row
    bitwise equal), as the paper's 4-row runs require."""
    nx, ny = 1024, 4
    f = workloads.progressive_wave(nx, ny, 2e-3, 0.4)
    with lbm.Grid(nx, ny, 0.6, 0.16, storage) as g:
        g.init(*f)
        g.step(300)
        rho, ux, uy = g.moments()
    for a in (rho, ux, uy):
        assert all(np.array_equal(a[0], a[y]) for y in range(1, ny))


@pytest.mark.parametrize("storage,tol", [("f32", 1e-6), ("f16d", 2e-5)])
@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 2), (1, 5), (5, 1), (2, 7), (7, 2), (3, 3), (8, 1)])
def test_tiny_grids_match_oracle(lbm, storage, tol, nx, ny):
    """Grids down to 1 x 1 (the periodic wrap makes x-1 and x+1 the same site
    or the site itself) match the oracle, through the step kernel (short
    calls) and the persistent launch (a long call)."""
    rng = np.random.default_rng(nx * 10 + ny)
    rho = 1 + 1e-3 * rng.standard_normal((ny, nx))
    ux = 1e-4 * rng.standard_normal((ny, nx))
    uy = 1e-4 * rng.standard_normal((ny, nx))
    tau, c2 = 0.8, 0.2
    with lbm.Grid(nx, ny, tau, c2, storage) as g:
        g.init(rho, ux, uy)
        g.step(3)
        g.step(70)
        got = g.moments()
    ref = oracle.simulate(rho, ux, uy, tau, c2, 73)
    err = max(np.abs(a - b).max() for a, b in zip(got, ref))
    assert err <= tol, err


@pytest.mark.parametrize("storage,tol", [("f32", 2e-9), ("f16d", 1e-6), ("bf16d", 1e-5)])
def test_init_then_moments_returns_the_fields(lbm, storage, tol):
    """The equilibrium of Eq. 2 has the moments of Eq. 3 exactly (sum w_i = 1,
    sum w_i e_i = 0, sum w_i e_i e_i = I/3), so moments right after init
    return the given fields up to the storage's rounding."""
    nx, ny = 300, 70
    rho, ux, uy = _fields(nx, ny, amp=1e-3, seed=21, u=1e-3)
    with lbm.Grid(nx, ny, 0.8, 0.2, storage) as g:
        g.init(rho, ux, uy)
        r, u, v = g.moments()
    err = max(np.abs(r - rho).max(), np.abs(u - ux).max(), np.abs(v - uy).max())
    assert err <= tol, err
