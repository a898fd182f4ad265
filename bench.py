"""Benchmark: MLUPS and fraction of the HBM roofline of the fused
variable-speed-of-sound D2Q9 step on one GB300 (or N replicas under torchrun).

Workload (N = 1): the 2048 x 2048 sweep: nine periodic FP32 grids with
c^2 = 0.05, 0.10, ..., 0.45, tau ~ U[0.55, 1.5] (seed 1), a standing acoustic
wave of amplitude log-spaced 1e-3 .. 5e-2 plus a shear wave
u_y = 1e-3 sin(2 pi x / nx).  One bench step = one time step of all nine grids
(9 launches of the step kernel).  Every grid's two buffers (2 x 151 MB) exceed
the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores on the same workload (one grid-step per bench step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0707_2437_gb300 import workloads  # noqa: E402

BYTES_PER_LU = {"f32": 72, "f16d": 36, "bf16d": 36}
METRIC = "MLUPS (million lattice updates per second), D2Q9 variable-speed-of-sound step"
WORKLOAD = "2048x2048 periodic D2Q9, 9 runs c2=0.05..0.45, tau~U[0.55,1.5], acoustic+shear wave"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "batch_sweep2048_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_0707_2437_gb300", "csrc", f)
                  for f in ("lbm_device.cuh", "lbm_kernels.cu", "lbm_batch_kernels.cuh")]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_setup(n_gpus: int):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.summarize(out.strip().splitlines())

    @staticmethod
    def summarize(lines):
        """Median and minimum SM clock, maximum clock, median power and the
        throttle reasons seen, from `--format=csv,noheader,nounits` lines of
        the query Q; None when no line parses."""
        sms, maxes, watts, reasons = [], [], [], set()
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxes.append(float(f[2]))
            except ValueError:
                continue
            try:
                watts.append(float(f[3]))
            except ValueError:
                pass
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes),
                "sm_min_mhz": min(sms),
                "power_w": statistics.median(watts) if watts else None,
                "samples": len(sms), "reasons": sorted(reasons)}


def serve_comparison(args, stream=None):
    """A serving trace (Poisson arrivals, mixed FP32 / FP16-delta requests)
    through the continuous-batching server and through the plain FIFO
    single-grid FP32 baseline: p50/p99 time-to-result and MLUPS, at the
    offered rate (above capacity: queueing included) and again with arrivals
    scaled to 0.7 of the server's measured capacity."""
    from paper_0707_2437_gb300 import serve
    trace = serve.scaled_trace(args.serve_count, args.serve_rate,
                               steps_hi=args.serve_steps_hi)
    overlap = not args.serve_no_overlap

    def server(schedule="lockstep", policy="fair"):
        return serve.Server(quantum=args.serve_quantum, overlap=overlap, schedule=schedule,
                            flow_updates=args.serve_flow_updates, policy=policy)

    warm = serve.scaled_trace(8, 1000.0, seed=99, hi=256, steps_hi=2000)
    server().run(warm, realtime=False)
    server("flow").run(warm, realtime=False)
    # The reference server steps every resident grid in lockstep.
    srv = server().run(trace, realtime=True).summary()
    out = {"trace": f"{args.serve_count} requests, Poisson {args.serve_rate}/s, sites "
                    f"log-uniform 128^2..2048^2, steps U{{1000..{args.serve_steps_hi}}}, "
                    "half f32 / half f16d",
           "admission": "overlapped with the running quantum" if overlap else "between quanta",
           "continuous_batching": srv, "fifo_f32": None}
    if not args.serve_skip_fifo:
        fifo = serve.serve_fifo(trace, realtime=True).summary()
        out.update({"fifo_f32": fifo,
                    "p99_speedup": fifo["p99_s"] / srv["p99_s"] if srv["p99_s"] else None,
                    "mlups_ratio": srv["mlups"] / fifo["mlups"] if fifo["mlups"] else None})
    # The same requests at 0.7 x the server's measured capacity (lattice
    # updates per second over the mean lattice updates of a request).
    mean_lu = float(np.mean([r.nx * r.ny * r.steps for r in trace]))
    rate07 = 0.7 * srv["mlups"] * 1e6 / mean_lu
    trace07 = serve.scaled_trace(args.serve_count, rate07, steps_hi=args.serve_steps_hi)
    srv07 = server().run(trace07, realtime=True).summary()
    out["at_0.7_capacity"] = {"rate_hz": rate07, "continuous_batching": srv07}
    if args.serve_srpt:
        # The same two traces, the grids with the least remaining work first.
        out["continuous_batching_srpt"] = server(policy="srpt").run(trace, realtime=True).summary()
        out["at_0.7_capacity"]["continuous_batching_srpt"] = server(policy="srpt").run(
            trace07, realtime=True).summary()
    # The same two traces with the flow schedule (each grid advances on its
    # own; launches share a budget of lattice updates by size^0.5), and with
    # the server's default: flow while at most 24 grids are resident,
    # lockstep above.
    for sched in ("flow", "auto"):
        if sched not in args.serve_schedules.split(","):
            continue
        name = f"continuous_batching_{sched}"
        out[name] = server(sched).run(trace, realtime=True).summary()
        out["at_0.7_capacity"][name] = server(sched).run(trace07, realtime=True).summary()
        out["flow_updates_per_launch"] = args.serve_flow_updates
    if not (args.serve_no_fifo07 or args.serve_skip_fifo):
        fifo07 = serve.serve_fifo(trace07, realtime=True).summary()
        out["at_0.7_capacity"]["fifo_f32"] = fifo07
        out["at_0.7_capacity"]["p99_speedup"] = (fifo07["p99_s"] / srv07["p99_s"]
                                                 if srv07["p99_s"] else None)
    return out


def sweep_fields(r):
    return workloads.acoustic_shear(r.nx, r.ny, r.amp)


def fourier_fields(r):
    return workloads.fourier_modes(r.nx, r.ny, amp=r.amp, seed=3)


FOURIER8192 = ("8192x8192 periodic D2Q9, tau=0.6, c2=0.15, rho = 1 + 8 seeded plane waves "
               "(integer wave numbers in [-4,4]^2, seed 3) scaled to max |rho - 1| = 1e-3, u = 0")


def cpu_baseline(seconds: float = 12.0, r=None, make_fields=sweep_fields):
    """The FP64 oracle as it stands, on the host cores, on one grid of the
    workload (the first 2048^2 grid of the sweep by default): runs whole
    steps until `seconds` have passed."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    r = r if r is not None else workloads.sweep_2048()[0]
    f = oracle.init(*make_fields(r))
    alpha = oracle.alpha_from_c2(r.c2)
    oracle.run(f, r.tau, alpha, 1)  # warm-up
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        oracle.run(f, r.tau, alpha, 1)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": r.nx * r.ny * steps / dt / 1e6, "unit": "MLUPS", "cores": used,
            "kind": "oracle",
            "sample": f"{steps} FP64 steps of one {r.nx}x{r.ny} grid of the workload "
                      f"({dt:.1f} s)"}


def sweep_config(storage: str, runs, workload_desc: str) -> dict:
    """`config` of the default line: the workload alone (sizes, storage, the
    L2 note), the same in the native and the reference arm."""
    state_mb = runs[0].nx * runs[0].ny * BYTES_PER_LU[storage] / 2 / 1e6  # one buffer
    return {"workload": workload_desc, "grids": len(runs), "nx": runs[0].nx, "ny": runs[0].ny,
            "storage": storage,
            "l2": (f"inputs larger than L2 (2 x {state_mb:.0f} MB per grid, 129 MB L2), "
                   "no flush")}


def run_reference(args):
    ws, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    from oracle import oracle
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    runs = workloads.sweep_2048()
    r = runs[0]
    f = oracle.init(*workloads.acoustic_shear(r.nx, r.ny, r.amp))
    for k in range(args.warmup):
        rr = runs[k % 9]
        oracle.run(f, rr.tau, oracle.alpha_from_c2(rr.c2), 1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        rr = runs[k % 9]
        oracle.run(f, rr.tau, oracle.alpha_from_c2(rr.c2), 1)
    dt = time.perf_counter() - t0
    value = r.nx * r.ny * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": sweep_config("f32", runs, WORKLOAD),
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": used, "kind": "oracle",
                         "sample": f"{args.steps} steps of one 2048x2048 grid, tau/c2 cycling "
                                   "through the 9 runs"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch

    from paper_0707_2437_gb300 import lbm

    ws, rank, local = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the native path has no CPU fallback)")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    if args.workload == "fourier8192":
        runs = [workloads.Run(8192, 8192, 0.6, 0.15, 1e-3)]
        make_fields, workload_desc = fourier_fields, FOURIER8192
    else:
        runs = workloads.sweep_2048()[:args.grids]
        make_fields, workload_desc = sweep_fields, WORKLOAD
    storage = args.storage
    if args.drive is not None:
        args.path = "single"  # batches refuse driven grids
    grids = []
    with torch.cuda.stream(stream):
        for r in runs:
            g = lbm.Grid(r.nx, r.ny, r.tau, r.c2, storage, stream=stream.cuda_stream)
            if args.c2_field:
                g.set_c2_field(workloads.c2_lens(r.nx, r.ny, r.c2))
            if args.drive is not None:
                g.set_drive(args.drive, 500.0)
            g.init(*make_fields(r))
            if args.config:
                g.set_config(*args.config)
            if args.rounding != "nearest":
                g.set_rounding(args.rounding)
            if args.stages is not None:
                g.set_pipeline(args.stages)
            grids.append(g)
    cfg = grids[0].get_config()
    stages, pipelined = grids[0].get_pipeline()
    sites = sum(r.nx * r.ny for r in runs)
    batch = lbm.Batch(grids) if args.path == "batch" else None
    if batch is not None and args.schedule != "lockstep":
        batch.set_schedule(args.schedule)
    if batch is not None and args.walk16:
        batch.set_walk16(args.walk16)
    if batch is not None and args.batch_rows:
        batch.set_config(args.batch_rows, 0)
    if batch is not None and args.tune:
        batch.tune()

    # Launch plan: on the batch path every launch is one persistent
    # cooperative kernel running `spl` steps of all grids (grid barrier between
    # steps), as lbm_batch_step runs a long call; the single-grid path launches
    # one step kernel per grid and step.
    spl = max(1, args.steps_per_launch) if batch is not None else 1

    def chunks(n):
        out = []
        while n > 0:
            out.append(min(spl, n))
            n -= out[-1]
        return out

    def advance(n):
        if batch is not None:
            batch.step(n)
        else:
            for g in grids:
                g.step(n)

    # Clock samples cover the warm-up, the timed region and about 1.2 s of the
    # same launches right after it (the timed region alone can be shorter than
    # nvidia-smi's 200 ms sample period).
    clocks = ClockSampler(local)
    clocks.start()
    for c in chunks(args.warmup):
        advance(c)
    torch.cuda.synchronize()

    # Timed region: events around every launch on the launching stream.
    plan = chunks(args.steps)
    per_step = 1 if batch is not None else len(grids)
    n_launch = len(plan) if batch is not None else args.steps * per_step
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_launch)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_launch)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    t_start.record(stream)
    k = 0
    if batch is not None:
        for c in plan:
            starts[k].record(stream)
            batch.step(c)
            ends[k].record(stream)
            k += 1
    else:
        for _ in range(args.steps):
            for g in grids:
                starts[k].record(stream)
                g.step(1)
                ends[k].record(stream)
                k += 1
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    t_pad = time.perf_counter()
    while time.perf_counter() - t_pad < args.clock_pad_s:
        advance(plan[0])
        torch.cuda.synchronize()
    clk = clocks.stop()
    if clk is not None:
        clk["window"] = (f"warm-up, the timed region and {args.clock_pad_s:.1f} s of the same "
                         "launches right after it")
    if batch is not None:
        batch.sync()
    elapsed_ms = t_start.elapsed_time(t_end)
    launch_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    elapsed_ms = max_over_ranks(ws, elapsed_ms)
    value = ws * sites * args.steps / (elapsed_ms * 1e-3) / 1e6

    # Roofline of the dominant kernel: algorithmic bytes of a launch / its
    # time, averaged over the launches (a launch = `spl` steps of all grids on
    # the batch path, one step of one grid on the single-grid path).
    # Algorithmic bytes of one launch's step: the distributions, plus the
    # 4-byte 1.5 alpha of every site with a c2 field, plus the drive's 27 ny
    # boundary stores.
    lu_bytes = BYTES_PER_LU[storage] + (4 if args.c2_field else 0)
    per_step_bytes = lu_bytes * (sites if batch is not None else runs[0].nx * runs[0].ny)
    b1 = lu_bytes * runs[0].nx * runs[0].ny  # one grid-step of the single-grid kernel
    if args.drive is not None and batch is None:
        per_step_bytes += 27 * runs[0].ny * (BYTES_PER_LU[storage] // 18)
    steps_launched = plan if batch is not None else [1] * n_launch
    achieved = per_step_bytes * sum(steps_launched) / (sum(launch_ms) * 1e-3) / 1e9
    per_launch_s = statistics.mean(launch_ms) * 1e-3
    alg_bytes = per_step_bytes * (spl if batch is not None else 1)
    peak, peak_kind = measured_peak()
    # The recorded traffic is that of the nine-grid sweep on the batch path.
    traffic = (recorded_traffic(storage, args.rounding, spl)
               if batch is not None and args.workload == "sweep2048" and len(runs) == 9
               and not args.c2_field else None)

    # The same batch with one step per launch, for the launch overhead, and
    # the plain single-grid step kernel on the same grids (one launch per grid
    # and step).  Both are timed as back-to-back sequences of launches with one
    # event pair around the sequence: the host enqueues faster than the GPU
    # runs, so the mean per launch is the kernel time plus the real gap between
    # kernels (events around each launch would also count the host's enqueue
    # latency, during which the GPU waits).
    def sequence_ms(n, launch):
        launch()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            launch()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    one_step = None
    if batch is not None and spl > 1:
        n1 = max(20, args.steps // 20)
        ms1 = sequence_ms(n1, lambda: batch.step(1))
        one_step = {"launches": n1, "mean_launch_ms": ms1,
                    "achieved": per_step_bytes / (ms1 * 1e-3) / 1e9,
                    "frac": per_step_bytes / (ms1 * 1e-3) / 1e9 / peak,
                    "mlups": sites / (ms1 * 1e-3) / 1e6,
                    "timing": "back-to-back launches, one event pair"}

    single = None
    if batch is not None and not args.no_single:
        n1 = max(20, args.steps // 10)

        def all_grids_one_step():
            for g in grids:
                g.step(1)

        ms1 = sequence_ms(n1, all_grids_one_step) / len(grids)
        single = {"kernel": f"k_step<{storage},vec={cfg[0]}>", "launches": n1 * len(grids),
                  "mean_launch_ms": ms1, "achieved": b1 / (ms1 * 1e-3) / 1e9,
                  "frac": b1 / (ms1 * 1e-3) / 1e9 / measured_peak()[0],
                  "mlups": runs[0].nx * runs[0].ny / (ms1 * 1e-3) / 1e6,
                  "timing": "back-to-back launches, one event pair"}

    # End to end through the C ABI with host buffers: one job = lbm_init from
    # pinned host fields, e2e_steps steps, lbm_moments back to pinned host
    # arrays, for all nine grids.
    n = runs[0].nx * runs[0].ny
    if args.no_e2e:
        args.e2e_jobs = 0
    e2e_runs = runs if args.e2e_jobs else []
    host_in = [[torch.from_numpy(a).pin_memory()
                for a in make_fields(r)] for r in e2e_runs]
    host_out = [[torch.empty((r.ny, r.nx), dtype=torch.float64).pin_memory() for _ in range(3)]
                for r in e2e_runs]

    def job(steps):
        for g, hin in zip(grids, host_in):
            g.init(*[t.numpy() for t in hin])
        if batch is not None:
            batch.step(steps)
        else:
            for g in grids:
                g.step(steps)
        for g, hout in zip(grids, host_out):
            g.moments(out=[t.numpy() for t in hout])

    # Pipelined jobs (batch path): a second set of grids on a stream of its
    # own, so that job j+1's input copies and job j-1's read-back run while
    # job j steps.  Every copy is still inside the timed region.
    pipelined = batch is not None and args.e2e_jobs > 1 and not args.e2e_serial
    sets = [(grids, batch)]
    if pipelined:
        stream_b = torch.cuda.Stream()
        grids_b = []
        for r in runs:
            g = lbm.Grid(r.nx, r.ny, r.tau, r.c2, storage, stream=stream_b.cuda_stream)
            if args.c2_field:
                g.set_c2_field(workloads.c2_lens(r.nx, r.ny, r.c2))
            if args.rounding != "nearest":
                g.set_rounding(args.rounding)
            grids_b.append(g)
        batch_b = lbm.Batch(grids_b)
        if args.schedule != "lockstep":
            batch_b.set_schedule(args.schedule)
        if args.walk16:
            batch_b.set_walk16(args.walk16)
        if args.batch_rows:
            batch_b.set_config(args.batch_rows, 0)
        sets.append((grids_b, batch_b))

    def init_set(k):
        for g, hin in zip(sets[k][0], host_in):
            g.init(*[t.numpy() for t in hin])

    # Device moments per set, then one copy to the pinned host arrays on a
    # side stream: the moments kernels are queued (and waited for) before the
    # next job's steps, so they do not queue behind that job's persistent
    # launch, and the copies to the host run while it steps.
    dev_out = ([[[torch.empty((r.ny, r.nx), dtype=torch.float64, device="cuda")
                  for _ in range(3)] for r in runs] for _ in range(2)] if pipelined else None)
    copy_stream = torch.cuda.Stream() if pipelined else None

    def moments_on_device(k):
        for g, dout in zip(sets[k][0], dev_out[k]):
            g.moments(out=dout)  # waits for the set's stream: its steps and this kernel

    def copy_out(k):
        with torch.cuda.stream(copy_stream):
            for dout, hout in zip(dev_out[k], host_out):
                for d_, h_ in zip(dout, hout):
                    h_.copy_(d_, non_blocking=True)
        copy_stream.synchronize()

    def pipelined_jobs(count, steps):
        init_set(0)
        sets[0][1].step(steps)
        for j in range(1, count):
            init_set(j % 2)              # host copies while job j-1 steps
            moments_on_device((j - 1) % 2)
            sets[j % 2][1].step(steps)
            copy_out((j - 1) % 2)        # device-to-host while job j steps
        moments_on_device((count - 1) % 2)
        copy_out((count - 1) % 2)

    if args.e2e_jobs:
        job(10)  # warm-up (graphs, allocator)
        if pipelined:
            pipelined_jobs(2, 10)
    e2e_clocks = ClockSampler(local)
    e2e_clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if pipelined:
        pipelined_jobs(args.e2e_jobs, args.e2e_steps)
    else:
        for _ in range(args.e2e_jobs):
            job(args.e2e_steps)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(ws, time.perf_counter() - t0)
    e2e_clk = e2e_clocks.stop()
    e2e_value = (ws * sites * args.e2e_steps * args.e2e_jobs / e2e_s / 1e6
                 if args.e2e_jobs else None)
    # One more job, outside the timed region, with a synchronisation after
    # each phase: where a job's time goes.
    e2e_phases = None
    if args.e2e_jobs:
        ta = time.perf_counter()
        for g, hin in zip(grids, host_in):
            g.init(*[t.numpy() for t in hin])
        for g in grids:
            g.sync()
        tb = time.perf_counter()
        if batch is not None:
            batch.step(args.e2e_steps)
            batch.sync()
        else:
            for g in grids:
                g.step(args.e2e_steps)
            for g in grids:
                g.sync()
        tc = time.perf_counter()
        for g, hout in zip(grids, host_out):
            g.moments(out=[t.numpy() for t in hout])
        td = time.perf_counter()
        e2e_phases = {"init_ms": 1e3 * (tb - ta), "steps_ms": 1e3 * (tc - tb),
                      "moments_ms": 1e3 * (td - tc)}

    job_bytes = len(runs) * 3 * n * 8  # rho, ux, uy in FP64, each way
    config = sweep_config(storage, runs, workload_desc)
    if args.c2_field:
        config["c2_field"] = "acoustic lens, c2 x (1 + 0.5 gaussian), 1.5 alpha per site in FP32"
    if args.drive is not None:
        config["drive"] = {"amplitude": args.drive, "period": 500.0}
    if args.rounding != "nearest":
        config["rounding"] = args.rounding
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if storage == "f32" else f"{storage} storage ({args.rounding} rounding), f32 math",
        "data": "synthetic",
        "config": config,
        "launch": {"tile": {"vec": cfg[0], "rows": cfg[1], "warps": cfg[2],
                            "pipeline_stages": stages if pipelined else 0},
                   "path": (f"persistent launches of {spl} steps over the {len(runs)} grid(s) "
                            "(batch API, grid barrier between steps)"
                            if batch is not None else "one step-kernel launch per grid and step"),
                   "steps_per_launch": spl,
                   "schedule": args.schedule if batch is not None else None,
                   "batch_config": batch.get_config() if batch is not None else None,
                   "batch_launch": batch.get_launch() if batch is not None else None,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "kernel": (f"k_batch_one (persistent, 9 grids, {spl} steps per launch)"
                                if batch is not None
                                else f"k_step_tma<{storage},stages={stages}>"
                                if pipelined and stages >= 2
                                else f"k_step<{storage},vec={cfg[0]}>"
                                + (" with c2 field" if args.c2_field else "")
                                + (" + k_drive_x" if args.drive is not None else "")),
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "mean_launch_ms": per_launch_s * 1e3},
        "e2e": {"value": e2e_value, "unit": "MLUPS",
                "h2d_bytes_per_step": job_bytes / args.e2e_steps,
                "d2h_bytes_per_step": job_bytes / args.e2e_steps,
                "h2d_bytes_per_job": job_bytes, "d2h_bytes_per_job": job_bytes,
                "steps_per_job": args.e2e_steps,
                "step": f"one job: lbm_init from pinned host fields, {args.e2e_steps} steps "
                        f"({'one batch launch' if batch is not None else 'lbm_step per grid'}), "
                        f"lbm_moments to host, for all {len(runs)} grids; the copies happen "
                        "once per job, so the bytes per step are the job's over its steps",
                "jobs": args.e2e_jobs, "phases_of_one_more_job": e2e_phases,
                "pipeline": ("two sets of grids on two streams: job j+1's lbm_init from host "
                             "fields and job j-1's read-back (lbm_moments into device arrays, "
                             "then a copy to pinned host arrays) overlap job j's steps"
                             if pipelined else "jobs one after another"),
                "clocks": e2e_clk},
        "gpu_launches": n_launch * (2 if args.drive is not None else 1),
        "clocks": clk,
        "single_grid_kernel": single,
        "batch_one_step_per_launch": one_step,
    }
    if batch is not None:
        batch.close()
    for g in grids:
        g.close()
    if pipelined:
        sets[1][1].close()
        for g in sets[1][0]:
            g.close()
    del grids, sets
    single_mlups = single["mlups"] if single else None
    if not args.no_legs and args.workload == "sweep2048" and not args.c2_field \
            and args.drive is None and storage == "f32":
        line["f16d_sweep"] = sweep_leg(args, "f16d", stream, single_mlups)
        line["batch512"] = {st: batch512_leg(args, st, stream, single_mlups)
                            for st in ("f32", "f16d")}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, runs[0], make_fields)
    if not args.no_serve:
        line["serve"] = serve_comparison(args, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)


def recorded_traffic(storage: str, rounding: str, spl: int):
    """DRAM bytes of one launch of `spl` steps of the nine-grid sweep on the
    batch path, from the ncu record under profiles/, or None when the record
    does not cover these kernel sources, this storage or this rounding."""
    if not os.path.exists(PROFILE_TRAFFIC) or rounding != "nearest":
        return None
    tj = json.load(open(PROFILE_TRAFFIC))
    entry = tj.get("storage", {}).get(storage)
    if entry and tj.get("source_hash") == kernel_source_hash() and tj.get("path") == "batch":
        # Captured on one-step launches of the same kernel; a launch of `spl`
        # steps makes the same accesses `spl` times.
        return entry["dram_bytes_per_step"] * spl
    return None


def sweep_leg(args, storage: str, stream, single_mlups):
    """The nine 2048^2 grids of the sweep in a 16-bit storage on the batch
    path, persistent launches of --steps-per-launch steps (CUDA events per
    launch on the launching stream): MLUPS, the roofline at that storage's
    algorithmic bytes, and the ratio over the plain FP32 single-grid kernel."""
    import torch

    from paper_0707_2437_gb300 import lbm
    runs = workloads.sweep_2048()
    spl = max(1, args.steps_per_launch)
    launches = max(1, args.leg_steps // spl)
    with torch.cuda.stream(stream):
        grids = []
        for r in runs:
            g = lbm.Grid(r.nx, r.ny, r.tau, r.c2, storage, stream=stream.cuda_stream)
            g.init(*sweep_fields(r))
            grids.append(g)
        b = lbm.Batch(grids)
        for _ in range(3):
            b.step(spl)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(launches)]
        for e0, e1 in ev:
            e0.record(stream)
            b.step(spl)
            e1.record(stream)
        torch.cuda.synchronize()
        status = b.sync()
        launch = b.get_launch()
        bcfg = b.get_config()
        b.close()
        for g in grids:
            g.close()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    sites = sum(r.nx * r.ny for r in runs)
    mlups = sites * spl * launches / (sum(ms) * 1e-3) / 1e6
    per_launch = BYTES_PER_LU[storage] * sites * spl
    achieved = per_launch / (statistics.mean(ms) * 1e-3) / 1e9
    peak, _ = measured_peak()
    return {"workload": "the nine 2048^2 grids of the sweep", "storage": storage,
            "rounding": "nearest", "steps": spl * launches, "steps_per_launch": spl,
            "mlups": mlups,
            "ratio_over_single_grid_kernel": mlups / single_mlups if single_mlups else None,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic(storage, "nearest", spl),
                         "bytes_per_update": BYTES_PER_LU[storage],
                         "kernel": f"k_batch_one<{storage}, vec {8 if storage != 'f32' else 4}>",
                         "algorithmic_bytes_per_launch": per_launch,
                         "mean_launch_ms": statistics.mean(ms)},
            "batch_config": bcfg, "batch_launch": launch, "batch_status": status}


def batch512_run(args, storage: str, rounding: str, steps: int, warmup: int, stream,
                 count: int = 512):
    """The 512 uneven grids (sites log-uniform 64^2 .. 1024^2, aspect
    2^U[-2, 2], per-grid tau and c^2) in one batch; `storage` is one kind or
    'mixed' (FP32 and FP16-delta in turn).  `steps` time steps of every grid
    in one lbm_batch_step call (one persistent launch per kind group, from a
    CUDA graph), timed with CUDA events on the batch's stream."""
    import torch

    from paper_0707_2437_gb300 import lbm
    runs = workloads.batch_grids(count)
    storages = [storage] if storage != "mixed" else ["f32", "f16d"]
    grids = []
    for k, r in enumerate(runs):
        st = storages[k % len(storages)]
        g = lbm.Grid(r.nx, r.ny, r.tau, r.c2, st, stream=stream.cuda_stream)
        if rounding != "nearest" and st != "f32":
            g.set_rounding(rounding)
        g.init(*workloads.sine_wave(r.nx, r.ny, r.amp, r.mode))
        grids.append(g)
    b = lbm.Batch(grids)
    if args.schedule != "lockstep":
        b.set_schedule(args.schedule)
    if args.batch_rows:
        b.set_config(args.batch_rows, 0)
    if args.walk16:
        b.set_walk16(args.walk16)
    if args.tune:
        b.tune()
    sites = sum(r.nx * r.ny for r in runs)
    alg = sum(r.nx * r.ny * lbm.BYTES_PER_LU[g.storage] for r, g in zip(runs, grids))
    b.step(warmup)
    b.sync()
    t0e = torch.cuda.Event(enable_timing=True)
    t1e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0e.record(stream)
    b.step(steps)
    t1e.record(stream)
    torch.cuda.synchronize()
    status = b.sync()
    ms = t0e.elapsed_time(t1e)
    out = {"ms": ms, "sites": sites, "alg_bytes_per_step": alg, "status": status,
           "batch_config": b.get_config(), "batch_launch": b.get_launch(),
           "grids": len(runs), "steps": steps}
    b.close()
    for g in grids:
        g.close()
    return out


def batch512_leg(args, storage: str, stream, single_mlups):
    """The 512-grid batch in one storage: MLUPS, roofline and the ratio over
    the plain FP32 single-grid kernel."""
    r = batch512_run(args, storage, "nearest", args.leg_steps, 5, stream)
    mlups = r["sites"] * r["steps"] / (r["ms"] * 1e-3) / 1e6
    achieved = r["alg_bytes_per_step"] * r["steps"] / (r["ms"] * 1e-3) / 1e9
    peak, _ = measured_peak()
    return {"workload": "batch of 512 uneven grids, sites log-uniform 64^2..1024^2, "
                        "aspect 2^U[-2,2]", "sites": r["sites"], "storage": storage,
            "steps": r["steps"], "launch": "one lbm_batch_step call of all steps",
            "mlups": mlups,
            "ratio_over_single_grid_kernel": mlups / single_mlups if single_mlups else None,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "bytes_per_update": BYTES_PER_LU[storage],
                         "algorithmic_bytes_per_step": r["alg_bytes_per_step"]},
            "batch_config": r["batch_config"], "batch_launch": r["batch_launch"],
            "batch_status": r["status"]}


def run_batch_workload(args):
    """512 uneven grids (64^2 .. 1024^2, aspect 2^U[-2,2]) stepped together:
    `--steps K` time steps of every grid in ONE persistent launch per kind
    group (replayed from a CUDA graph), after `--warmup` steps."""
    import torch

    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    r = batch512_run(args, args.storage, args.rounding, args.steps, args.warmup, stream,
                     args.batch_count)
    barrier(ws)
    clk = clocks.stop()
    ms = max_over_ranks(ws, r["ms"])
    value = ws * r["sites"] * args.steps / (ms * 1e-3) / 1e6
    achieved = r["alg_bytes_per_step"] * args.steps / (ms * 1e-3) / 1e9
    peak, _ = measured_peak()
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.storage} storage, f32 math", "data": "synthetic",
        "config": {"workload": f"batch of {r['grids']} uneven grids, sites log-uniform "
                               "64^2..1024^2, aspect 2^U[-2,2]",
                   "sites": r["sites"], "storage": args.storage, "rounding": args.rounding,
                   "schedule": args.schedule,
                   "l2": f"working set {r['alg_bytes_per_step'] / 1e9:.1f} GB >> 129 MB L2, "
                         "no flush"},
        "launch": {"batch_config": r["batch_config"], "batch_launch": r["batch_launch"],
                   "path": "one lbm_batch_step call of all steps: one persistent cooperative "
                           "launch per kind group"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_batch_one / k_batch",
                     "algorithmic_bytes_per_step": r["alg_bytes_per_step"]},
        "gpu_launches": r["batch_config"]["groups"], "clocks": clk, "batch_status": r["status"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_slab_workload(args):
    """One grid split along y between the ranks (one GPU each): every step
    is the local step of each rank's slab and the halo exchange (two rows of
    all nine planes with each neighbour, NCCL point-to-point; with one rank,
    the slab's own rows wrap around).  Strong scaling: the grid is fixed."""
    import functools

    import torch

    from paper_0707_2437_gb300 import lbm, slab

    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    n = args.slab_n
    if n % ws:
        raise SystemExit(f"bench.py: the {n} rows do not split evenly over {ws} ranks")
    ny_local = n // ws
    tau, c2 = 0.6, 0.15
    rho, ux, uy = workloads.fourier_modes(n, n, amp=1e-3, seed=3)
    rows = [(rank * ny_local - 2 + k) % n for k in range(ny_local + 4)]
    stream = torch.cuda.current_stream()
    s = lbm.Slab(n, ny_local, tau, c2, args.storage, stream=stream)
    s.init(rho[rows], ux[rows], uy[rows])
    del rho, ux, uy
    ds = slab.DeviceSlab(s)
    runner = slab.SlabRunner(ds, functools.partial(slab.exchange, rank=rank, world=ws))
    runner.run(args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ds.step()
        runner.refresh()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = max_over_ranks(ws, e0.elapsed_time(e1))
    value = n * n * args.steps / (ms * 1e-3) / 1e6
    per_rank_bytes = BYTES_PER_LU[args.storage] * n * ny_local * args.steps
    achieved = per_rank_bytes / (ms * 1e-3) / 1e9
    peak, _ = measured_peak()
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": "f32" if args.storage == "f32" else f"{args.storage} storage, f32 math",
        "data": "synthetic",
        "config": {"workload": f"one {n}x{n} periodic grid split in y over the ranks, tau={tau}, "
                               f"c2={c2}, 8 seeded plane waves of amplitude 1e-3",
                   "storage": args.storage, "rows_per_rank": ny_local,
                   "l2": f"{2 * n * (ny_local + 4) * BYTES_PER_LU[args.storage] / 2 / 1e9:.1f} GB "
                         "of state per rank, no flush"},
        "launch": {"path": "lbm_step(1) per slab (the batch kernel over the own rows) and a "
                           "halo exchange per step", "halo_bytes_per_side": s.halo_bytes,
                   "parallelism": f"slabs x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "note": "per rank: the algorithmic bytes of its own rows over the step time "
                             "including the exchange"},
        "gpu_launches": args.steps, "clocks": clk,
    }
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve_workload(args):
    """The serving trace through the continuous-batching server and through
    the plain FIFO single-grid FP32 baseline; p50/p99 time-to-result and
    aggregate MLUPS of both."""
    import torch

    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    clocks = ClockSampler(local)
    clocks.start()
    cmp_ = serve_comparison(args)
    srv, fifo = cmp_["continuous_batching"], cmp_["fifo_f32"]
    clk = clocks.stop()
    line = {
        "metric": "served p50/p99 time-to-result and aggregate MLUPS vs plain FP32 FIFO",
        "value": srv["mlups"], "unit": "MLUPS", "n_gpus": ws, "steps": args.serve_count,
        "warmup": 8, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "half f32, half f16d storage, f32 math", "data": "synthetic",
        "config": {"workload": f"{args.serve_count} Poisson requests at {args.serve_rate}/s, "
                               f"sites log-uniform 128^2..2048^2, steps U{{1000..{args.serve_steps_hi}}}",
                   "quantum_steps": args.serve_quantum},
        "served": srv, "fifo_f32": fifo, "at_0.7_capacity": cmp_["at_0.7_capacity"],
        "served_flow": cmp_.get("continuous_batching_flow"),
        "served_auto": cmp_.get("continuous_batching_auto"),
        "served_srpt": cmp_.get("continuous_batching_srpt"),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--storage", default="f32", choices=list(BYTES_PER_LU) + ["mixed"])
    ap.add_argument("--workload", default="sweep2048",
                    choices=["sweep2048", "fourier8192", "batch", "serve", "slab"])
    ap.add_argument("--rounding", default="nearest", choices=["nearest", "stochastic"],
                    help="rounding of 16-bit stores")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--slab-n", type=int, default=8192,
                    help="side of the grid the slab workload splits over the ranks")
    ap.add_argument("--batch-rows", type=int, default=0)
    ap.add_argument("--walk16", default=None, choices=["auto", "v8", "v4", "v4pf2"],
                    help="walk of 16-bit grids in batch kernels (default: the library's)")
    ap.add_argument("--c2-field", action="store_true",
                    help="per-site c2 (an acoustic lens) on every grid")
    ap.add_argument("--drive", type=float, default=None,
                    help="driven channel with this amplitude (period 500); single-grid path")
    ap.add_argument("--steps-per-launch", type=int, default=20,
                    help="steps of all grids per persistent launch on the batch path")
    ap.add_argument("--tune", action="store_true")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving comparison in the default workload")
    ap.add_argument("--serve-count", type=int, default=60)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-steps-hi", type=int, default=5000)
    ap.add_argument("--serve-quantum", type=int, default=256)
    ap.add_argument("--schedule", default="lockstep", choices=["lockstep", "flow"],
                    help="batch schedule on the batch paths (flow: no barrier across grids)")
    ap.add_argument("--serve-srpt", action="store_true",
                    help="also run the least-remaining-work-first server in the serving comparison")
    ap.add_argument("--serve-schedules", default="flow,auto",
                    help="server schedules run beside lockstep in the serving comparison "
                         "(comma-separated: flow, auto; empty for none)")
    ap.add_argument("--serve-flow-updates", type=float, default=1e9,
                    help="lattice updates per launch shared by the flow-schedule server")
    ap.add_argument("--serve-no-overlap", action="store_true",
                    help="admit requests between quanta instead of during them")
    ap.add_argument("--serve-skip-fifo", action="store_true",
                    help="skip the FIFO baseline at both rates")
    ap.add_argument("--serve-no-fifo07", action="store_true",
                    help="skip the FIFO baseline at 0.7x the server's capacity (long traces)")
    ap.add_argument("--config", type=int, nargs=3, default=None,
                    metavar=("VEC", "ROWS", "WARPS"))
    ap.add_argument("--stages", type=int, default=None,
                    help="row pipeline stages (0: register walk)")
    ap.add_argument("--path", default="batch", choices=["batch", "single"],
                    help="batch: one persistent launch per step over all grids; "
                         "single: one step-kernel launch per grid and step")
    ap.add_argument("--no-single", action="store_true",
                    help="skip the extra single-grid kernel measurement")
    ap.add_argument("--grids", type=int, default=9, choices=range(1, 10),
                    help="use the first N of the nine 2048^2 runs (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--e2e-jobs", type=int, default=3)
    ap.add_argument("--e2e-serial", action="store_true",
                    help="run the e2e jobs one after another (no second set of grids)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the FP16-delta sweep and 512-grid batch legs of the default run")
    ap.add_argument("--leg-steps", type=int, default=200,
                    help="time steps timed in each extra leg")
    ap.add_argument("--clock-pad-s", type=float, default=1.2,
                    help="seconds of the same launches run after the timed region while "
                         "the clocks are sampled")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_workload(args)
    elif args.workload == "serve":
        run_serve_workload(args)
    elif args.workload == "slab":
        run_slab_workload(args)
    else:
        if args.storage == "mixed":
            ap.error("--storage mixed applies to the batch workload")
        run_native(args)


if __name__ == "__main__":
    main()
