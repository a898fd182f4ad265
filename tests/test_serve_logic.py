"""Host logic of the continuous-batching server, on the CPU: the device layer
(grids, batches, free memory) is replaced by a fake that keeps the same
bookkeeping, so admission by free memory, slot limits, arrival order, the
per-grid step limits and retirement are checked without a GPU."""
import pytest

from paper_0707_2437_gb300 import serve, workloads


class _FakeDevice:
    def __init__(self, total):
        self.total = total
        self.used = 0
        self.live = 0
        self.max_live = 0
        self.max_used = 0
        self.created = []
        self.in_flight = None    # the batch whose quantum is queued, until sync
        self.streams = 0
        self.steps = []          # (schedule, [(sites, steps)]) of every step call

    # the subset of the lbm module the server uses
    def load(self):
        return None

    def mem_info(self):
        return self.total - self.used, self.total

    def bytes_required(self, nx, ny, storage):
        return nx * ny * (72 if storage == "f32" else 36)


def _fake_lbm(dev):
    class Grid:
        def __init__(self, nx, ny, tau, c2, storage="f32", stream=None):
            self.nx, self.ny, self.storage = nx, ny, storage
            self.stream = stream
            self.made_in_flight = dev.in_flight is not None
            self.bytes = dev.bytes_required(nx, ny, storage)
            dev.used += self.bytes
            dev.max_used = max(dev.max_used, dev.used)
            dev.live += 1
            dev.max_live = max(dev.max_live, dev.live)
            dev.created.append(self)
            self.t = 0
            self.closed = False
            self.steps_at_close = None

        def init(self, rho, ux, uy):
            assert rho.shape == (self.ny, self.nx)

        def moments(self):
            assert dev.in_flight is None
            return (None, None, None)

        def set_stream(self, stream):
            self.stream = stream

        def sync(self):
            pass

        def close(self):
            assert not self.closed
            self.closed = True
            self.steps_at_close = self.t
            dev.used -= self.bytes
            dev.live -= 1

    class Batch:
        def __init__(self, grids):
            assert all(not g.closed for g in grids)
            assert dev.in_flight is None
            self.grids = list(grids)
            self.stream = self.grids[0].stream
            assert all(g.stream is self.stream for g in self.grids)

        def set_schedule(self, schedule):
            assert schedule in ("lockstep", "flow")
            self.schedule = schedule

        def step(self, n, limits=None):
            assert dev.in_flight is None
            limits = limits or [n] * len(self.grids)
            for g, lim in zip(self.grids, limits):
                assert 0 <= lim <= n
                g.t += lim
            dev.steps.append((getattr(self, "schedule", "lockstep"),
                              [(g.nx * g.ny, lim) for g, lim in zip(self.grids, limits)]))
            dev.in_flight = self

        def sync(self):
            dev.in_flight = None
            return 0

        def close(self):
            pass

    ns = type("FakeLbm", (), {})()
    ns.load, ns.mem_info, ns.bytes_required = dev.load, dev.mem_info, dev.bytes_required
    ns.Grid, ns.Batch = Grid, Batch

    def new_stream():
        dev.streams += 1
        return object()

    ns.new_stream = new_stream
    return ns


def _requests(n=12, seed=7):
    return workloads.serve_trace(count=n, rate_hz=1000.0, seed=seed, lo=64, hi=256,
                                 steps_lo=100, steps_hi=1500)


def test_every_request_runs_exactly_its_steps(monkeypatch):
    dev = _FakeDevice(total=1 << 40)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    reqs = _requests()
    stats = serve.Server(quantum=256, reserve_bytes=0, schedule="lockstep").run(reqs, realtime=False)
    assert sorted(r.rid for r in stats.results) == [q.rid for q in reqs]
    by_rid = {g_rid: g for g_rid, g in zip([q.rid for q in reqs], dev.created)}
    for q in reqs:
        assert by_rid[q.rid].steps_at_close == q.steps
    assert dev.live == 0 and dev.used == 0
    assert stats.lattice_updates == sum(q.steps * q.nx * q.ny for q in reqs)
    longest = max(q.steps for q in reqs)
    assert stats.quanta >= -(-longest // 256)


def test_admission_is_bounded_by_free_memory(monkeypatch):
    reqs = _requests()
    need = max(serve.Server(reserve_bytes=0)._need(q) for q in reqs)
    reserve = 1000
    dev = _FakeDevice(total=reserve + 2 * need + need // 2)  # room for two at a time
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    stats = serve.Server(quantum=128, reserve_bytes=reserve, schedule="lockstep").run(
        reqs, realtime=False)
    assert len(stats.results) == len(reqs)
    assert dev.max_live >= 2 and stats.max_active == dev.max_live
    assert dev.max_used <= dev.total - reserve   # the reserve is never touched
    assert dev.max_live < len(reqs)             # memory, not the trace, set the bound
    assert dev.used == 0


def test_slot_limit_and_arrival_order(monkeypatch):
    dev = _FakeDevice(total=1 << 40)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    reqs = _requests(n=10)
    stats = serve.Server(quantum=64, reserve_bytes=0, max_slots=3, schedule="lockstep").run(
        reqs, realtime=False)
    assert stats.max_active == 3 and dev.max_live == 3
    admitted = sorted(stats.results, key=lambda r: (r.admitted_s, r.rid))
    assert [r.rid for r in admitted] == sorted(r.rid for r in stats.results)
    assert all(r.arrival_s == 0.0 for r in stats.results)  # all present at time 0


def test_request_larger_than_the_device_is_refused(monkeypatch):
    reqs = _requests(n=3)
    dev = _FakeDevice(total=10)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    with pytest.raises(MemoryError):
        serve.Server(quantum=64, reserve_bytes=0, schedule="lockstep").run(reqs, realtime=False)


def test_summary_percentiles():
    st = serve.ServeStats()
    for k in range(100):
        st.results.append(serve.Result(k, 0.0, 0.0, float(k + 1), 10, 100, "f32"))
    st.makespan_s = 100.0
    st.lattice_updates = 1000
    s = st.summary()
    assert s["requests"] == 100
    assert abs(s["p50_s"] - 50.5) < 1e-9 and 98.9 < s["p99_s"] < 99.1
    assert s["mlups"] == pytest.approx(1e-5)


@pytest.mark.parametrize("overlap", [True, False])
def test_admission_overlaps_the_running_quantum(monkeypatch, overlap):
    """With overlap, requests that arrive while a quantum runs are created
    during it, on the batch's own stream (not the legacy default stream), and
    join at the next quantum; every batch holds grids of one stream.  Without
    overlap nothing is created while a quantum is queued."""
    dev = _FakeDevice(total=1 << 40)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    reqs = _requests(n=12)
    srv = serve.Server(quantum=64, reserve_bytes=0, max_slots=4, overlap=overlap,
                       schedule="lockstep")
    stats = srv.run(reqs, realtime=False)
    assert len(stats.results) == len(reqs) and dev.live == 0
    made = [g.made_in_flight for g in dev.created]
    assert any(made) == overlap
    assert dev.streams == (1 if overlap else 0)
    if overlap:
        assert all(g.stream is not None for g in dev.created)
    for q, g in zip(reqs, dev.created):
        assert g.steps_at_close == q.steps


def test_flow_schedule_shares_updates_equally(monkeypatch):
    """With the flow schedule every launch gives each resident grid about the
    same number of lattice updates (steps in inverse proportion to its size,
    at least one, at most its remaining steps and the per-launch cap), and
    every request still runs exactly its steps."""
    dev = _FakeDevice(total=1 << 40)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    reqs = _requests(n=16)
    budget = 4e6
    srv = serve.Server(reserve_bytes=0, schedule="flow", flow_updates=budget, flow_max_steps=900,
                       flow_weight=0.0)
    stats = srv.run(reqs, realtime=False)
    assert len(stats.results) == len(reqs) and dev.live == 0
    for q, g in zip(reqs, dev.created):
        assert g.steps_at_close == q.steps
    assert dev.steps and all(sch == "flow" for sch, _ in dev.steps)
    for _, calls in dev.steps:
        share = budget / len(calls)
        for sites, lim in calls:
            assert 1 <= lim <= 900
            # at most the share, unless a single step already exceeds it
            assert lim * sites <= max(share, sites)
    # small grids took more steps per launch than large ones in a shared launch
    _, first = dev.steps[0]
    by_size = sorted(first)
    assert by_size[0][1] >= by_size[-1][1]


def test_auto_schedule_switches_with_the_resident_count(monkeypatch):
    """'auto' steps in the flow schedule while few grids are resident and in
    lockstep once more than auto_grids are; requests still run their steps."""
    dev = _FakeDevice(total=1 << 40)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    reqs = _requests(n=16)
    stats = serve.Server(reserve_bytes=0, schedule="auto", auto_grids=6).run(reqs, realtime=False)
    assert len(stats.results) == len(reqs) and dev.live == 0
    for q, g in zip(reqs, dev.created):
        assert g.steps_at_close == q.steps
    scheds = {(sch, len(calls) > 6) for sch, calls in dev.steps}
    assert ("lockstep", True) in scheds and ("flow", False) in scheds
    assert ("flow", True) not in scheds and ("lockstep", False) not in scheds


def test_unknown_schedule_is_refused():
    with pytest.raises(ValueError):
        serve.Server(schedule="eager")


def test_srpt_policy_steps_the_least_remaining_work_first(monkeypatch):
    """The srpt policy steps, in each launch, the grids with the least
    remaining work until their sites reach the threshold (at least one grid);
    the others take no steps.  Every request still completes its steps."""
    dev = _FakeDevice(total=1 << 40)
    monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
    reqs = _requests(n=16)
    thresh = 3 * 128 * 128
    srv = serve.Server(quantum=128, reserve_bytes=0, policy="srpt", srpt_sites=thresh,
                       schedule="lockstep")
    stats = srv.run(reqs, realtime=False)
    assert len(stats.results) == len(reqs) and dev.live == 0
    for q, g in zip(reqs, dev.created):
        assert g.steps_at_close == q.steps
    paused_seen = False
    for _, calls in dev.steps:
        stepping = [s for s, lim in calls if lim > 0]
        assert stepping
        # the stepping grids, minus the last one added, stay below the threshold
        assert sum(stepping) - max(stepping) < thresh or len(stepping) == 1
        paused_seen = paused_seen or any(lim == 0 for _, lim in calls)
    assert paused_seen


def test_unknown_policy_is_refused():
    with pytest.raises(ValueError):
        serve.Server(policy="lifo")


def test_flow_shares_weighted_by_size(monkeypatch):
    """With flow_weight w a grid's share of a launch's updates is in
    proportion to sites^w: w = 1 gives every grid the same steps (up to what
    it has left), w = 0.5 gives larger grids more updates but fewer steps."""
    for w in (1.0, 0.5):
        dev = _FakeDevice(total=1 << 40)
        monkeypatch.setattr(serve, "lbm", _fake_lbm(dev))
        reqs = _requests(n=12)
        srv = serve.Server(reserve_bytes=0, schedule="flow", flow_updates=2e7,
                           flow_max_steps=10 ** 6, flow_weight=w)
        srv.run(reqs, realtime=False)
        _, first = dev.steps[0]
        wts = [s_ ** w for s_, _ in first]
        for (sites, lim), wt in zip(first, wts):
            share = 2e7 * wt / sum(wts)
            assert lim <= max(1, share // sites)
        by_size = sorted(first)
        if w == 0.5:
            assert by_size[0][1] >= by_size[-1][1]
            assert by_size[0][0] * by_size[0][1] <= by_size[-1][0] * by_size[-1][1] * 1.01 + by_size[-1][0]
