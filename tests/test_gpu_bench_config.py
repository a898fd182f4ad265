"""Parity at full size in the launch configuration the benchmark times: the
nine 2048^2 grids of the sweep in one batch, persistent launches of 20 steps
(the default line in FP32, the f16d_sweep leg in FP16-delta storage).  Every
site of the smallest- and the largest-amplitude grid after two launches
against the FP64 oracle run of the same steps (batch and solo runs are
bitwise equal for every grid, tested elsewhere).

Bounds.  FP32: each step rounds about twenty operations per site on stored
values of at most about 5 A, adding as a random walk over n steps:
sqrt(n) * 100 * 2^-24 * A.  FP16-delta: every stored h_i is rounded to 11
significant bits (half a unit: 2^-12 of |h| <= 5 A), about ten stores feed a
moment, adding as a random walk: sqrt(n) * 10 * 2^-12 * 5 A."""
import numpy as np
import pytest

from oracle import oracle
from paper_0707_2437_gb300 import workloads

pytestmark = pytest.mark.gpu

_REF = {}


@pytest.mark.parametrize("storage", ["f32", "f16d"])
def test_sweep_batch_launches_match_oracle(lbm, storage):
    runs = workloads.sweep_2048()
    grids = []
    for r in runs:
        g = lbm.Grid(r.nx, r.ny, r.tau, r.c2, storage)
        g.init(*workloads.acoustic_shear(r.nx, r.ny, r.amp))
        grids.append(g)
    b = lbm.Batch(grids)
    steps, spl = 40, 20
    for _ in range(steps // spl):
        b.step(spl)
    assert b.sync() == 0
    assert b.get_launch()["last"] == "graph"
    got = {j: grids[j].moments() for j in (0, 8)}
    b.close()
    for g in grids:
        g.close()
    oracle.set_threads(0)
    for j in (0, 8):
        r = runs[j]
        if j not in _REF:
            _REF[j] = oracle.simulate(*workloads.acoustic_shear(r.nx, r.ny, r.amp), r.tau, r.c2,
                                      steps)
        err = max(float(np.abs(a - c).max()) for a, c in zip(got[j], _REF[j]))
        if storage == "f32":
            tol = np.sqrt(steps) * 100 * 2.0 ** -24 * r.amp
        else:
            tol = np.sqrt(steps) * 10 * 2.0 ** -12 * 5 * r.amp
        print(f"{storage} grid {j} (A = {r.amp:.3g}): max |GPU - oracle| = {err:.2e} (bound {tol:.2e})")
        assert err <= tol
