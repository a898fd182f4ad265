"""Batched and served forms on the GPU: each result in the mix equals the
same request run alone (bitwise: the batch kernel does the single-grid
kernel's arithmetic in the same order)."""
import numpy as np
import pytest

from paper_0707_2437_gb300 import lbm as _lbm_mod
from paper_0707_2437_gb300 import serve, workloads

pytestmark = pytest.mark.gpu


def _trace():
    specs = [(64, 64, "f32", 120), (96, 40, "f16d", 300), (128, 128, "bf16d", 80),
             (40, 72, "f32", 200), (256, 32, "f16d", 64), (72, 24, "f32", 150),
             (37, 29, "f32", 90)]
    rng = np.random.default_rng(12)
    return [workloads.Request(rid=k, arrival_s=0.01 * k, nx=nx, ny=ny,
                              tau=float(rng.uniform(0.55, 1.2)),
                              c2=float(rng.uniform(0.05, 0.4)), steps=steps, storage=st)
            for k, (nx, ny, st, steps) in enumerate(specs)]


@pytest.mark.parametrize("overlap,schedule,policy", [(True, "lockstep", "fair"),
                                                     (False, "lockstep", "fair"),
                                                     (True, "lockstep", "srpt"),
                                                     (True, "flow", "fair"),
                                                     (True, "flow", "srpt"),
                                                     (True, "auto", "fair")])
def test_served_results_equal_solo_runs(lbm, overlap, schedule, policy):
    reqs = _trace()
    srv = serve.Server(quantum=48, max_slots=3, keep_fields=True, reserve_bytes=0,
                       overlap=overlap, schedule=schedule, policy=policy,
                       flow_updates=2e5, flow_max_steps=64, srpt_sites=8000, auto_grids=2)
    stats = srv.run(reqs, realtime=False)
    assert len(stats.results) == len(reqs)
    assert stats.max_active == 3
    assert stats.quanta > 3
    # Later requests joined the running set when earlier ones finished.
    first_done = min(r.finished_s for r in stats.results)
    assert any(r.admitted_s >= first_done for r in stats.results)
    by_id = {r.rid: r for r in stats.results}
    for req in reqs:
        with lbm.Grid(req.nx, req.ny, req.tau, req.c2, req.storage) as g:
            g.init(*serve._fields(req))
            g.step(req.steps)
            solo = g.moments()
        got = by_id[req.rid].fields
        for a, b in zip(got, solo):
            assert np.array_equal(a, b), req
    s = stats.summary()
    assert s["p99_s"] >= s["p50_s"] > 0


def test_fifo_baseline_runs(lbm):
    reqs = _trace()[:3]
    stats = serve.serve_fifo(reqs, realtime=False)
    assert [r.rid for r in stats.results] == [0, 1, 2]
    assert stats.summary()["mlups"] > 0


@pytest.mark.parametrize("kind", ["f16d", "bf16d", "f16d-sr", "bf16d-sr"])
@pytest.mark.parametrize("rows", [1, 5, 16])
def test_batch_walk16_variants_bitwise_equal(lbm, kind, rows):
    """The walks of 16-bit grids (8 sites per lane; 4 per lane with one or two
    rows of loads in flight; the automatic choice) leave the same state bit
    for bit, for tile heights down to a single row; a grid with nx a multiple
    of 4 but not 8 takes the 4-site walk within the 8-site setting."""
    sizes = [(256, 40), (128, 33), (64, 7), (36, 12)]
    out = {}
    for walk in ("auto", "v8", "v4", "v4pf2"):
        grids = []
        for nx, ny in sizes:
            g = lbm.Grid(nx, ny, 0.7, 0.2, kind.replace("-sr", ""))
            if kind.endswith("-sr"):
                g.set_rounding("stochastic")
            g.init(*workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny))
            grids.append(g)
        b = lbm.Batch(grids)
        b.set_config(rows, 0)
        b.set_walk16(walk)
        assert b.get_config()["walk16"] == walk
        b.step(37)
        assert b.sync() == 0
        out[walk] = [g.get_state()[0] for g in grids]
        b.close()
        for g in grids:
            g.close()
    for w in ("auto", "v4", "v4pf2"):
        for a, c in zip(out["v8"], out[w]):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("kind", ["f16d", "bf16d-sr"])
def test_batch_walk16_single_kind_specialised(lbm, kind):
    """A batch of one 16-bit kind runs one specialised launch in every walk."""
    for walk in ("auto", "v8", "v4", "v4pf2"):
        g = lbm.Grid(512, 64, 0.8, 0.2, kind.replace("-sr", ""))
        if kind.endswith("-sr"):
            g.set_rounding("stochastic")
        g.init(*workloads.fourier_modes(512, 64, amp=1e-3, seed=2))
        b = lbm.Batch([g])
        b.set_walk16(walk)
        cfg = b.get_config()
        assert cfg["specialised"] and cfg["groups"] == 1
        b.step(3)
        assert b.sync() == 0
        b.close()
        g.close()


def test_batch_walk16_argument_checks(lbm):
    g = lbm.Grid(64, 8, 0.8, 0.2, "f16d")
    b = lbm.Batch([g])
    for bad in (4, -1):
        assert b.lib.lbm_batch_set_walk16(b.b, bad) == lbm.LBM_EINVAL
    with pytest.raises(KeyError):
        b.set_walk16("v16")
    b.close()
    g.close()


def test_kind_groups_equal_solo_runs(lbm):
    """A batch whose FP32 and FP16-D grids each fill the GPU runs them in
    separate specialised launches (with the small odd-width grid in a launch of
    the general kernel): 3 kind groups, and every grid reaches bitwise the
    state it reaches alone, including per-grid step limits."""
    specs = [(2048, 2048, 0.8, 0.2, "f32"), (2048, 2048, 0.6, 0.1, "f16d"),
             (37, 29, 0.7, 0.3, "f32"), (256, 64, 0.9, 0.25, "bf16d")]
    limits = [12, 9, 12, 5]
    solo = []
    for (nx, ny, tau, c2, st), lim in zip(specs, limits):
        with lbm.Grid(nx, ny, tau, c2, st) as g:
            g.init(*workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny))
            g.step(lim)
            solo.append(g.get_state()[0])
    grids = []
    for nx, ny, tau, c2, st in specs:
        g = lbm.Grid(nx, ny, tau, c2, st)
        g.init(*workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny))
        grids.append(g)
    b = lbm.Batch(grids)
    assert b.get_config()["groups"] == 3
    b.step(7, limits)
    b.step(5, [max(0, x - 7) for x in limits])
    assert b.sync() == 0
    for g, s, lim in zip(grids, solo, limits):
        assert g.t == lim
        assert np.array_equal(g.get_state()[0], s)
    b.close()
    for g in grids:
        g.close()


def test_batch_tune_leaves_state_and_results_unchanged(lbm):
    """lbm_batch_tune times dry one-step runs over tile heights and 16-bit
    walks: the grids' states and step counts are unchanged (so is the
    stochastic-rounding stream, keyed by the step), the chosen
    configuration is one of the candidates, and stepping afterwards gives the
    same state bit for bit as an untuned batch."""
    specs = [(512, 128, "f32"), (256, 96, "f16d"), (136, 40, "bf16d")]
    out = {}
    for tuned in (False, True):
        grids = []
        for nx, ny, st in specs:
            g = lbm.Grid(nx, ny, 0.8, 0.2, st)
            g.init(*workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx))
            if st == "bf16d":
                g.set_rounding("stochastic")
            grids.append(g)
        b = lbm.Batch(grids)
        if tuned:
            before = [g.get_state() for g in grids]
            cfg = b.tune()
            assert cfg["rows"] in (8, 12, 16, 24, 32)
            assert cfg["walk16"] in ("auto", "v8", "v4", "v4pf2")
            for g, (s0, t0) in zip(grids, before):
                s1, t1 = g.get_state()
                assert t1 == t0 == 0 and np.array_equal(s0, s1)
        b.step(25)
        assert b.sync() == 0
        out[tuned] = [g.get_state()[0] for g in grids]
        b.close()
        for g in grids:
            g.close()
    for a, c in zip(out[False], out[True]):
        assert np.array_equal(a, c)


def test_batch_orders_with_members_streams(lbm):
    """Grids initialised on streams of their own are batched on another
    stream: the batch waits for their initialisation, and moments read on a
    member's own stream right after the step call (no batch sync) see the
    batch's result.  The heavy first grid keeps the batch's stream busy, so
    a missing wait would show."""
    specs = [(2048, 1024, "f32"), (256, 96, "f16d"), (192, 64, "f32")]
    streams = [lbm.new_stream() for _ in specs]
    grids, solo = [], []
    for (nx, ny, st), s in zip(specs, streams):
        fields = workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny)
        with lbm.Grid(nx, ny, 0.7, 0.25, st) as g:
            g.init(*fields)
            g.step(40)
            solo.append(g.moments())
        g = lbm.Grid(nx, ny, 0.7, 0.25, st, stream=s)
        g.init(*fields)
        grids.append(g)
    b = lbm.Batch(grids)
    b.step(40)
    got = [g.moments() for g in grids[::-1]]
    for a, c in zip(got[::-1], solo):
        for x, y in zip(a, c):
            assert np.array_equal(x, y)
    assert b.sync() == 0
    b.close()
    for g in grids:
        g.close()


def test_set_stream_keeps_order(lbm):
    """A grid initialised on one stream and moved to another steps from its
    initial state; moving it again between step calls changes nothing."""
    nx, ny = 1024, 512
    fields = workloads.fourier_modes(nx, ny, amp=1e-3, seed=5)
    with lbm.Grid(nx, ny, 0.8, 0.2, "f16d") as g:
        g.init(*fields)
        g.step(300)
        ref = g.moments()
    s1, s2 = lbm.new_stream(), lbm.new_stream()
    with lbm.Grid(nx, ny, 0.8, 0.2, "f16d", stream=s1) as g:
        g.init(*fields)
        g.set_stream(s2)
        g.step(100)            # persistent launch on s2
        g.set_stream(s1)       # waits for it, drops the persistent batch
        g.step(200)
        got = g.moments()
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_batch_replays_from_cuda_graph(lbm):
    """The default launch mode replays the batch's persistent launches from a
    CUDA graph on this GPU (no capture failure), and the graph, forced-graph
    and direct modes give bitwise the same states."""
    specs = [(512, 256, 0.8, 0.2, "f32"), (256, 96, 0.6, 0.1, "f16d"), (37, 29, 0.7, 0.3, "f32")]

    def run(mode):
        grids = []
        for nx, ny, tau, c2, st in specs:
            g = lbm.Grid(nx, ny, tau, c2, st)
            g.init(*workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx))
            grids.append(g)
        b = lbm.Batch(grids)
        assert b.get_launch() == {"mode": "auto", "last": None, "capture_failed": False}
        if mode != "auto":
            b.set_launch(mode)
        b.step(20)
        b.step(20)
        assert b.sync() == 0
        info = b.get_launch()
        states = [g.get_state()[0] for g in grids]
        b.close()
        for g in grids:
            g.close()
        return info, states

    auto, s_auto = run("auto")
    assert auto == {"mode": "auto", "last": "graph", "capture_failed": False}
    forced, s_graph = run("graph")
    assert forced["last"] == "graph"
    direct, s_direct = run("direct")
    assert direct == {"mode": "direct", "last": "direct", "capture_failed": False}
    for a, b_, c in zip(s_auto, s_graph, s_direct):
        assert np.array_equal(a, b_) and np.array_equal(a, c)


def test_batch_launch_mode_argument_checks(lbm):
    g = lbm.Grid(64, 64, 0.8, 0.2)
    g.init(*workloads.sine_wave(64, 64))
    b = lbm.Batch([g])
    for bad in (-1, 3):
        assert b.lib.lbm_batch_set_launch(b.b, bad) == lbm.LBM_EINVAL
    with pytest.raises(KeyError):
        b.set_launch("eager")
    b.close()
    g.close()


def _solo_states(lbm, specs, limits, fields_of, rounding=None):
    out = []
    for (nx, ny, tau, c2, st), lim in zip(specs, limits):
        with lbm.Grid(nx, ny, tau, c2, st) as g:
            if rounding and st != "f32":
                g.set_rounding(rounding)
            g.init(*fields_of(nx, ny))
            g.step(lim)
            out.append(g.get_state()[0])
    return out


@pytest.mark.parametrize("rows", [16, 5, 1])
def test_flow_schedule_equals_solo_runs(lbm, rows):
    """The flow schedule (no barrier across the batch; each tile waits only
    for the tiles it reads from) gives every grid bitwise the state it reaches
    alone: mixed storages and walks, per-grid step limits, odd widths (1-site
    lanes), single-row tail segments (rows 5 with ny = 41, and rows 1) and
    grids down to 1 x 1, over two calls."""
    specs = [(2048, 512, 0.8, 0.2, "f32"), (1024, 256, 0.6, 0.1, "f16d"),
             (37, 41, 0.7, 0.3, "f32"), (256, 40, 1.1, 0.3, "bf16d"),
             (96, 130, 0.55, 0.05, "f16d"), (8, 8, 0.9, 0.4, "f32"), (1, 1, 0.9, 0.2, "f32"),
             (3, 5, 0.7, 0.15, "f16d"), (520, 16, 0.7, 0.25, "f32")]
    limits = [30, 80, 200, 45, 120, 200, 7, 150, 1]

    def fields(nx, ny):
        return workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx * 7 + ny)

    solo = _solo_states(lbm, specs, limits, fields)
    grids = []
    for nx, ny, tau, c2, st in specs:
        g = lbm.Grid(nx, ny, tau, c2, st)
        g.init(*fields(nx, ny))
        grids.append(g)
    b = lbm.Batch(grids)
    b.set_config(rows, 0)
    b.set_schedule("flow")
    assert b.get_schedule() == "flow"
    b.step(120, limits)
    b.step(80, [max(0, x - 120) for x in limits])
    assert b.sync() == 0
    for g, s, lim in zip(grids, solo, limits):
        assert g.t == lim
        assert np.array_equal(g.get_state()[0], s)
    b.close()
    for g in grids:
        g.close()


def test_flow_schedule_stochastic_rounding_and_graph(lbm):
    """Stochastic rounding seeds by each grid's own step counter, so the flow
    schedule reproduces solo runs bitwise with it too; repeated calls with
    the same step count replay the captured graph."""
    specs = [(512, 128, 0.7, 0.2, "f16d"), (264, 40, 0.9, 0.1, "bf16d"), (40, 24, 0.6, 0.3, "f32")]
    limits = [64, 40, 64]

    def fields(nx, ny):
        return workloads.fourier_modes(nx, ny, amp=1e-2, seed=nx + 3)

    solo = _solo_states(lbm, specs, limits, fields, rounding="stochastic")
    grids = []
    for nx, ny, tau, c2, st in specs:
        g = lbm.Grid(nx, ny, tau, c2, st)
        if st != "f32":
            g.set_rounding("stochastic")
        g.init(*fields(nx, ny))
        grids.append(g)
    b = lbm.Batch(grids)
    b.set_schedule("flow")
    for _ in range(4):
        b.step(16, [16, 10, 16])
    assert b.get_launch()["last"] == "graph"
    assert b.sync() == 0
    for g, s, lim in zip(grids, solo, limits):
        assert g.t == lim
        assert np.array_equal(g.get_state()[0], s)
    b.close()
    for g in grids:
        g.close()


def test_flow_schedule_timeout_reports_status(lbm):
    """A 1-microsecond wait limit runs out in the flow schedule too (a tile
    waiting for its neighbours): the kernel ends, the host reads
    LBM_ETIMEOUT, and a later call with the normal limit succeeds."""
    grids = [lbm.Grid(1024, 1024, 0.8, 0.2) for _ in range(2)]
    for g in grids:
        g.init(*workloads.sine_wave(1024, 1024))
    b = lbm.Batch(grids)
    b.set_schedule("flow")
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


def test_flow_schedule_serving_mix_two_walks(lbm):
    """The serving mix (FP32 and FP16-delta grids, nx multiples of 8) runs
    the flow kernel with both walks inlined; every grid equals its solo run
    bitwise, including grids small enough for short tiles."""
    specs = [(2048, 256, 0.8, 0.2, "f32"), (512, 512, 0.6, 0.1, "f16d"),
             (128, 128, 0.7, 0.3, "f32"), (136, 72, 0.9, 0.25, "f16d"), (64, 8, 0.55, 0.05, "f16d")]
    limits = [20, 60, 300, 250, 90]

    def fields(nx, ny):
        return workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx + ny)

    solo = _solo_states(lbm, specs, limits, fields)
    grids = []
    for nx, ny, tau, c2, st in specs:
        g = lbm.Grid(nx, ny, tau, c2, st)
        g.init(*fields(nx, ny))
        grids.append(g)
    b = lbm.Batch(grids)
    b.set_schedule("flow")
    assert b.get_config()["specialised"]
    b.step(300, limits)
    assert b.sync() == 0
    for g, s_, lim in zip(grids, solo, limits):
        assert g.t == lim
        assert np.array_equal(g.get_state()[0], s_)
    b.close()
    for g in grids:
        g.close()
