"""The split walk.  A lockstep batch of 8-site 16-bit grids pairs the tiles of
its grids at most 128 columns wide (when they are at least a fifth of its
tiles): two consecutive segments share one warp, a half-warp each.  Each grid
must end bit for bit in the state the single-grid step kernel gives it alone
(the same per-site arithmetic in the same order), and in the FP64 oracle's
state within the storage's bound."""
import numpy as np
import pytest

from oracle import oracle
from paper_0707_2437_gb300 import workloads

pytestmark = pytest.mark.gpu

# Grids 8, 40, 128, 96 and 120 columns wide pair; 136, 200, 264 and 384 stay
# single walks (wider than a half-warp's 128 columns), in the same kernel.
# Heights give one segment, even and odd counts, and a last segment of one
# row.
SIZES = [(8, 40), (40, 17), (128, 33), (136, 64), (264, 24), (384, 50), (96, 8), (120, 31),
         (200, 20)]


def _expected_pairs(nx, ny, rows):
    return (-(-ny // rows)) // 2 if nx <= 128 else 0


def _make(lbm, kind, nx, ny, k):
    g = lbm.Grid(nx, ny, 0.55 + 0.05 * k, 0.05 + 0.03 * k, kind.replace("-sr", ""))
    if kind.endswith("-sr"):
        g.set_rounding("stochastic")
    g.init(*workloads.fourier_modes(nx, ny, amp=1e-2, seed=7 * k + 1))
    return g


@pytest.mark.parametrize("kind", ["f16d", "bf16d", "f16d-sr", "bf16d-sr"])
@pytest.mark.parametrize("rows", [16, 5, 1])
def test_split_walk_equals_single_grid_kernel(lbm, kind, rows):
    limits = [30, 30, 23, 30, 30, 11, 30, 30, 30]
    grids = [_make(lbm, kind, nx, ny, k) for k, (nx, ny) in enumerate(SIZES)]
    b = lbm.Batch(grids)
    b.set_config(rows, 0)
    cfg = b.get_config()
    assert cfg["specialised"] and cfg["groups"] == 1
    assert cfg["paired_tiles"] == sum(_expected_pairs(nx, ny, rows) for nx, ny in SIZES)
    assert cfg["paired_tiles"] > 0
    b.step(30, limits)
    assert b.sync() == 0
    got = [g.get_state()[0] for g in grids]
    b.close()
    for g in grids:
        g.close()
    for k, ((nx, ny), lim) in enumerate(zip(SIZES, limits)):
        with _make(lbm, kind, nx, ny, k) as h:
            h.set_persistent(False)
            h.step(lim)
            solo = h.get_state()[0]
        assert np.array_equal(got[k], solo), (kind, rows, nx, ny)


@pytest.mark.parametrize("storage,tol", [("f16d", 2e-5), ("bf16d", 2e-4)])
def test_split_walk_matches_oracle(lbm, storage, tol):
    """A 120 x 45 grid (three segments: a pair and a single walk) and a
    384 x 40 grid (single walks in the same kernel) against the FP64 oracle
    after 200 steps at amplitude 1e-3, within the 16-bit bounds of the
    single-grid parity test."""
    specs = [(120, 45, 0.6, 0.15), (384, 40, 0.9, 0.3)]
    fields = [workloads.fourier_modes(nx, ny, amp=1e-3, seed=nx) for nx, ny, _, _ in specs]
    grids = []
    for (nx, ny, tau, c2), f in zip(specs, fields):
        g = lbm.Grid(nx, ny, tau, c2, storage)
        g.init(*f)
        grids.append(g)
    b = lbm.Batch(grids)
    cfg = b.get_config()  # the default configuration: short tiles for a small batch
    assert cfg["paired_tiles"] == _expected_pairs(120, 45, cfg["rows"]) > 0
    b.step(200)
    assert b.sync() == 0
    for g, (nx, ny, tau, c2), f in zip(grids, specs, fields):
        got = g.moments()
        ref = oracle.simulate(*f, tau, c2, 200)
        err = max(np.abs(a - r).max() for a, r in zip(got, ref))
        print(f"{storage} {nx}x{ny}: max |GPU - oracle| = {err:.3e}")
        assert err <= tol
    b.close()
    for g in grids:
        g.close()


def test_no_pairs_outside_single_kind_lockstep(lbm):
    """FP32 grids, 16-bit grids on the 4-site walk, mixed kinds in the general
    kernel, the 'v8' walk setting and the flow schedule walk every tile
    alone."""
    cases = [
        [("f32", 120, 40)],
        [("f16d", 124, 40)],                       # nx not a multiple of 8: 4-site walk
        [("f16d", 120, 40), ("f32", 64, 16)],      # mixed kinds, small: general kernel
        [("f16d", 2048, 64), ("f16d", 120, 40)],   # narrow tiles 3 of 35: under a fifth
        [("f16d", 264, 48)],                       # a narrow last strip of a wider grid
    ]
    for spec in cases:
        grids = [lbm.Grid(nx, ny, 0.7, 0.2, st) for st, nx, ny in spec]
        for g in grids:
            g.init(*workloads.sine_wave(g.nx, g.ny, 1e-3))
        b = lbm.Batch(grids)
        assert b.get_config()["paired_tiles"] == 0, spec
        b.close()
        for g in grids:
            g.close()
    g = lbm.Grid(120, 40, 0.7, 0.2, "f16d")
    g.init(*workloads.sine_wave(120, 40, 1e-3))
    b = lbm.Batch([g])
    want = _expected_pairs(120, 40, b.get_config()["rows"])
    assert b.get_config()["paired_tiles"] == want > 0
    b.set_walk16("v8")
    assert b.get_config()["paired_tiles"] == 0
    b.set_walk16("auto")
    assert b.get_config()["paired_tiles"] == want
    b.set_schedule("flow")
    assert b.get_config()["paired_tiles"] == 0
    b.close()
    g.close()
