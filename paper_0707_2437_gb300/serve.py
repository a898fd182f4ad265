"""Continuous-batching serving loop for variable-speed-of-sound simulations.

Requests (grid size, tau, c^2, step count, storage) arrive over time.  The
server keeps every admitted grid's distributions resident in HBM and advances
all of them together with the batch API (one persistent launch per quantum of
steps, each grid limited to its remaining steps).  While a quantum runs it
admits waiting requests, in arrival order, as long as the free device memory
(lbm_mem_info) minus a reserve covers the new grid (lbm_bytes_required plus the
staging of its initial fields) and a slot is free; their grids are created and
initialised meanwhile and join at the next quantum.  After each quantum it retires
finished grids (their moments are the result) and frees their memory.  So
requests that arrive while others are on the GPU join the running set as
memory frees up, and their work overlaps on the device.

``serve_fifo`` is the plain baseline: one grid at a time, in arrival order,
with the single-grid FP32 kernel.

Schedules (``Server(schedule=...)``).  ``lockstep``: each launch advances
every resident grid by up to `quantum` steps together, a barrier across the
batch between steps, so a small grid waits as many batch-wide steps as a large
one.  ``flow``: each launch shares a budget of lattice updates equally between
the grids (a small grid gets many steps, a large one few) and runs them with
the batch's flow schedule, where each grid advances on its own.  ``auto``:
flow while at most `auto_grids` grids are resident, lockstep above.

Two policies (``Server(policy=...)``) pick the grids that step in a launch:
``fair`` steps every resident grid; ``srpt`` steps the grids with the least
remaining work first (shortest remaining processing time), adding grids until
their sites keep the GPU's memory bandwidth busy, while the others wait.

All stepping runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lbm, workloads


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    sites: int
    storage: str
    fields: tuple | None = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    makespan_s: float = 0.0
    lattice_updates: int = 0
    quanta: int = 0
    max_active: int = 0
    # Host wall time by phase: grid creation and initial fields ("admit"),
    # batch (re)creation and queueing the quantum ("batch"), waiting for the
    # quantum to finish ("step"), retirement: results and frees ("retire").
    phase_s: dict = field(default_factory=lambda: {"admit": 0.0, "batch": 0.0,
                                                   "step": 0.0, "retire": 0.0})

    def summary(self) -> dict:
        lat = np.array([r.latency_s for r in self.results]) if self.results else np.zeros(1)
        return {
            "requests": len(self.results),
            "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()),
            "makespan_s": self.makespan_s,
            "mlups": self.lattice_updates / self.makespan_s / 1e6 if self.makespan_s else 0.0,
            "quanta": self.quanta,
            "max_active": self.max_active,
            "phase_s": dict(self.phase_s),
        }


def _fields(req: workloads.Request):
    m = 1 + req.rid % 3
    return workloads.sine_wave(req.nx, req.ny, req.amp, m)


class Server:
    """Continuous batching over the batch API.

    With ``overlap=True`` (the default) the batch runs on a stream of its own
    and arriving requests are admitted while a quantum runs: their grids are
    created on the batch's stream and initialised there.  lbm_init copies host
    fields on the library's copy stream and returns once they are read, with
    the initialisation kernel queued behind the running quantum, so the host's
    field set-up and the copies overlap the kernel.  The new grids join the
    batch at the next quantum.  With ``overlap=False`` admission happens
    between quanta, on ``stream``."""

    def __init__(self, quantum: int = 256, reserve_bytes: int = 4 << 30,
                 max_slots: int = 512, keep_fields: bool = False, stream=None,
                 overlap: bool = True, schedule: str = "auto",
                 flow_updates: float = 1e9, flow_max_steps: int = 1024,
                 flow_weight: float = 0.5, policy: str = "fair", srpt_sites: float = 4e6,
                 auto_grids: int = 24):
        self.quantum = quantum
        self.reserve = reserve_bytes
        self.max_slots = max_slots
        self.keep_fields = keep_fields
        self.stream = stream
        self.overlap = overlap
        if schedule not in ("lockstep", "flow", "auto"):
            raise ValueError(f"unknown schedule {schedule!r}")
        self.schedule = schedule
        self.auto_grids = auto_grids
        self.flow_updates = flow_updates
        self.flow_max_steps = flow_max_steps
        self.flow_weight = flow_weight
        if policy not in ("fair", "srpt"):
            raise ValueError(f"unknown policy {policy!r}")
        self.policy = policy
        self.srpt_sites = srpt_sites
        lbm.load()

    def _selected(self, active):
        """Which resident grids step in the next launch.  'fair': all of
        them.  'srpt': the grids with the least remaining work (steps left
        times sites), smallest first, until their sites reach `srpt_sites`
        (enough for a step to be bound by memory bandwidth rather than by the
        walk of one tile); the rest wait with a step limit of 0."""
        if self.policy == "fair":
            return [True] * len(active)
        order = sorted(range(len(active)), key=lambda j: active[j][2] * active[j][0].nx
                       * active[j][0].ny)
        sel = [False] * len(active)
        sites = 0
        for j in order:
            sel[j] = True
            sites += active[j][0].nx * active[j][0].ny
            if sites >= self.srpt_sites:
                break
        return sel

    def _schedule_for(self, active) -> str:
        """'auto': the flow schedule while at most `auto_grids` grids are
        resident (each grid's time-to-result then follows its own size), the
        lockstep schedule above (a backlog: throughput sets the latencies)."""
        if self.schedule != "auto":
            return self.schedule
        return "flow" if len(active) <= self.auto_grids else "lockstep"

    def _limits(self, active, schedule=None):
        """Steps each resident grid takes in the next launch.  Lockstep:
        every grid up to `quantum` steps (all advance together).  Flow: the
        launch's budget of `flow_updates` lattice updates is shared between
        the grids in proportion to sites^flow_weight (0: equally, so a grid
        takes steps in inverse proportion to its size; 1: in proportion to
        its size, every grid the same steps), at least one step, at most
        `flow_max_steps` and what the grid has left; the flow schedule runs
        them without a barrier across grids."""
        sel = self._selected(active)
        run = [a for a, s_ in zip(active, sel) if s_]
        if (schedule or self._schedule_for(active)) == "lockstep":
            q = min(self.quantum, max(a[2] for a in run))
            return q, [min(q, a[2]) if s_ else 0 for a, s_ in zip(active, sel)]
        wts = [(a[0].nx * a[0].ny) ** self.flow_weight for a in run]
        total_w = sum(wts)
        lim, j = [], 0
        for a, s_ in zip(active, sel):
            if not s_:
                lim.append(0)
                continue
            share = self.flow_updates * wts[j] / total_w
            j += 1
            lim.append(int(min(a[2], self.flow_max_steps, max(1, share // (a[0].nx * a[0].ny)))))
        return max(lim), lim

    def _need(self, req) -> int:
        # distributions + the staging of three FP64 fields during lbm_init
        return lbm.bytes_required(req.nx, req.ny, req.storage) + 24 * req.nx * req.ny

    def run(self, requests, realtime: bool = True) -> ServeStats:
        """Serves `requests` (sorted by arrival).  With realtime=True arrivals
        follow the wall clock from the start of the call; otherwise every
        request is present at time 0."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        active = []  # [req, grid, remaining, admitted_s]
        stats = ServeStats()
        ph = stats.phase_s
        batch = None
        batch_sched = "lockstep"
        members = None
        main = self.stream
        if self.overlap and main is None:
            # Not the legacy default stream: that one would make the copies
            # and host calls around the running quantum wait for it.
            main = lbm.new_stream()
        t0 = time.perf_counter()
        i = 0

        def now():
            return time.perf_counter() - t0

        def admit(incoming):
            # Admit arrived requests, in order, while memory and slots allow.
            nonlocal i
            ta = time.perf_counter()
            free, _ = lbm.mem_info()
            while i < len(pending) and len(active) + len(incoming) < self.max_slots:
                req = pending[i]
                if realtime and req.arrival_s > now():
                    break
                need = self._need(req)
                if need > free - self.reserve:
                    if not active and not incoming:
                        raise MemoryError(f"request {req.rid} needs {need} bytes, "
                                          f"{free} free")
                    break
                g = lbm.Grid(req.nx, req.ny, req.tau, req.c2, req.storage, stream=main)
                g.init(*_fields(req))
                incoming.append([req, g, req.steps, now()])
                free -= need
                i += 1
            ph["admit"] += time.perf_counter() - ta

        while i < len(pending) or active:
            incoming = []
            if not self.overlap:
                admit(incoming)
                active += incoming
                incoming = []
            # Queue one quantum for the resident grids (asynchronous).
            limits = None
            if active:
                tb = time.perf_counter()
                sched = self._schedule_for(active)
                if batch is None or members != [id(a[1]) for a in active]:
                    if batch is not None:
                        batch.close()
                    batch = lbm.Batch([a[1] for a in active])
                    batch_sched = "lockstep"
                    members = [id(a[1]) for a in active]
                if sched != batch_sched:
                    batch.set_schedule(sched)
                    batch_sched = sched
                stats.max_active = max(stats.max_active, len(active))
                q, limits = self._limits(active, sched)
                batch.step(q, limits)
                ph["batch"] += time.perf_counter() - tb
            if self.overlap:
                admit(incoming)  # while the quantum is on the GPU

            if limits is not None:
                ts = time.perf_counter()
                batch.sync()
                tr = time.perf_counter()
                ph["step"] += tr - ts
                stats.quanta += 1
                for a, lim in zip(active, limits):
                    a[2] -= lim
                    stats.lattice_updates += lim * a[0].nx * a[0].ny
                keep = []
                for a in active:
                    req, g, rem, adm = a
                    if rem > 0:
                        keep.append(a)
                        continue
                    fields = g.moments() if self.keep_fields else None
                    if not self.keep_fields:
                        g.sync()
                    arrival = req.arrival_s if realtime else 0.0
                    stats.results.append(Result(req.rid, arrival, adm, now(), req.steps,
                                                req.nx * req.ny, req.storage, fields))
                    g.close()
                if len(keep) != len(active):
                    batch.close()
                    batch = None
                    members = None
                active = keep
                ph["retire"] += time.perf_counter() - tr
            active += incoming
            if not active and i < len(pending):
                # Idle until the next arrival.
                wait = pending[i].arrival_s - now()
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        if batch is not None:
            batch.close()
        stats.makespan_s = now()
        return stats


def serve_fifo(requests, realtime: bool = True, storage: str = "f32",
               keep_fields: bool = False, stream=None) -> ServeStats:
    """Plain baseline: each request alone, in arrival order, single-grid
    kernel, stored as `storage` (FP32 by default) whatever it asked for.
    With realtime=False every request is present at time 0."""
    lbm.load()
    stats = ServeStats()
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival_s):
        if realtime:
            wait = req.arrival_s - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        start = time.perf_counter() - t0
        with lbm.Grid(req.nx, req.ny, req.tau, req.c2, storage, stream=stream) as g:
            g.init(*_fields(req))
            g.step(req.steps)
            fields = g.moments() if keep_fields else None
            if not keep_fields:
                g.sync()
        arrival = req.arrival_s if realtime else 0.0
        stats.results.append(Result(req.rid, arrival, start, time.perf_counter() - t0,
                                    req.steps, req.nx * req.ny, storage, fields))
        stats.lattice_updates += req.steps * req.nx * req.ny
        stats.max_active = 1
    stats.makespan_s = time.perf_counter() - t0
    return stats


def scaled_trace(count: int, rate_hz: float, seed: int = 5, **kw):
    """The serving trace with a chosen arrival rate (for a load below capacity)."""
    return workloads.serve_trace(count=count, rate_hz=rate_hz, seed=seed, **kw)
