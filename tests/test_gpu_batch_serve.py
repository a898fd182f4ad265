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


def test_served_results_equal_solo_runs(lbm):
    reqs = _trace()
    srv = serve.Server(quantum=48, max_slots=3, keep_fields=True, reserve_bytes=0)
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
