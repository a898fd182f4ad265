"""Element-wise parity with the FP64 oracle on the long and large runs: the
paper's viscous-decay runs down to tau = 0.501 (Section 4, Eq. 10, Fig. 6),
the damping run at alpha = -0.65 (Section 4, Fig. 5), the large-amplitude runs
of the 2048^2 sweep on the whole grid, and a slice of the 512-grid batch with
mixed storages in one batched call.

Tolerance of an FP32 run of n steps.  Each step rounds about twenty FP32
operations per site on stored values of at most about 5 A (A the density
amplitude of the wave; the stored h_i are of the size of the deviation), each
to 2^-24 of its size.  The acoustic and shear modes these runs carry are
damped by less than 1 % over the run at the smallest tau, so their rounding
adds up as a random walk: sqrt(n) * 20 * 2^-24 * 5 A.  The bound asserted is
that, rounded up: sqrt(n) * 100 * 2^-24 * A, on every site's rho, u_x and u_y.

16-bit storages round every stored h_i (FP16: 2^-11, BF16: 2^-8 relative);
their bounds are those of the 500-step parity test of the same amplitude
(FP16-delta 2e-5, BF16-delta 2e-4), doubled with stochastic rounding (a stored
value is off by up to one unit in the last place instead of a half).
"""
import numpy as np
import pytest

from oracle import oracle
from paper_0707_2437_gb300 import workloads

pytestmark = pytest.mark.gpu


def _f32_bound(steps: int, amp: float) -> float:
    return np.sqrt(steps) * 100 * 2.0 ** -24 * amp


def _max_err(got, ref):
    return max(float(np.abs(a - b).max()) for a, b in zip(got, ref))


def _mode1(field):
    """|mode 1 in x| of a [ny, nx] field (2/N sum v e^{-2 pi i x/nx})."""
    ny, nx = field.shape
    ph = 2 * np.pi * np.arange(nx)[None, :] / nx
    c = 2.0 / field.size * (field * np.cos(ph)).sum()
    s = 2.0 / field.size * (field * np.sin(ph)).sum()
    return float(np.hypot(c, s))


@pytest.mark.parametrize("tau", [0.501, 0.55])
def test_decay_run_matches_oracle(lbm, tau):
    """The viscous-decay run of Section 4 (Eq. 10, Fig. 6): wave (2)-type
    progressive wave, alpha = -0.6, lambda = 400, 100 periods (41,408 steps)
    on a 400 x 4 grid, at tau = 0.501 (the most rounding-sensitive setting:
    1/tau = 1.996) and 0.55.  Every site's moments against the oracle run of
    the same steps, and the decay ratio of Eq. 10 from both."""
    lam, alpha, u0 = 400, -0.6, 1e-5
    c2 = 1 / 3 - alpha
    ce = np.sqrt(c2)
    steps = int(round(100 * lam / ce))
    f = workloads.progressive_wave(lam, 4, u0, ce)
    with lbm.Grid(lam, 4, tau, c2) as g:
        g.init(*f)
        g.step(steps)
        got = g.moments()
    fo = oracle.init(*f)
    oracle.run(fo, tau, alpha, steps)
    ref = oracle.moments(fo)
    amp = u0 / ce
    err = _max_err(got, ref)
    tol = _f32_bound(steps, amp)
    ratio_gpu = _mode1(got[1]) / u0
    ratio_ora = _mode1(ref[1]) / u0
    print(f"tau={tau}: {steps} steps, max |GPU - oracle| = {err:.2e} (bound {tol:.2e}); "
          f"A/A0 GPU {ratio_gpu:.6f}, oracle {ratio_ora:.6f}")
    assert err <= tol
    assert abs(ratio_gpu - ratio_ora) <= tol / amp


def test_damping_run_alpha_minus_065_matches_oracle(lbm):
    """The damping run of Section 4 (Fig. 5) at its most negative alpha,
    -0.65, tau = 0.52, lambda = 400: 2000 steps, a one-period window of
    16 samples, 40,000 steps, a second window.  The GPU's window amplitudes
    and final state against the oracle's on the same schedule, and the decay
    rate per step between the windows from both."""
    lam, tau, u0, alpha = 400, 0.52, 1e-5, -0.65
    c2 = 1 / 3 - alpha
    ce = np.sqrt(c2)
    period = lam / ce
    dt = int(round(period / 16))
    f = workloads.progressive_wave(lam, 4, u0, ce)
    schedule = [2000] + [dt] * 16 + [40000 - 16 * dt] + [dt] * 16

    gpu_amps = []
    with lbm.Grid(lam, 4, tau, c2) as g:
        g.init(*f)
        for n in schedule:
            g.step(n)
            gpu_amps.append(float(np.hypot(*g.mode("ux", 1, 0))))
        got = g.moments()
    ora_amps = []
    fo = oracle.init(*f)
    for n in schedule:
        oracle.run(fo, tau, alpha, n)
        ora_amps.append(_mode1(oracle.moments(fo)[1]))
    ref = oracle.moments(fo)
    steps = sum(schedule)
    amp = u0 / ce
    tol = _f32_bound(steps, amp)
    err = _max_err(got, ref)
    a_gpu, a_ora = np.array(gpu_amps), np.array(ora_amps)
    # Window means (the first window ends at sample 17, the second at 34).
    span = sum(schedule[1:18])
    rate_gpu = -np.log(a_gpu[18:].mean() / a_gpu[1:17].mean()) / span
    rate_ora = -np.log(a_ora[18:].mean() / a_ora[1:17].mean()) / span
    print(f"alpha=-0.65: {steps} steps, max |GPU - oracle| = {err:.2e} (bound {tol:.2e}); "
          f"rate GPU {rate_gpu:.6e}, oracle {rate_ora:.6e}")
    assert err <= tol
    assert np.abs(a_gpu - a_ora).max() <= tol
    # Each window mean is within tol of the oracle's, so the log ratio of the
    # two windows, and with it rate * span, is within 2 tol / (smaller mean).
    a_min = min(a_ora[1:17].mean(), a_ora[18:].mean())
    assert abs(rate_gpu - rate_ora) * span <= 2 * tol / a_min


@pytest.mark.parametrize("run", [7, 8])
def test_large_amplitude_sweep_runs_whole_grid(lbm, run):
    """The two largest-amplitude runs of the 2048^2 sweep (A = 3.1e-2 and
    5e-2, c^2 = 0.40 and 0.45, plus the shear wave), where the waves are no
    longer linear: every site's moments after 1000 steps (lbm_step's
    persistent launch) against a 1000-step oracle run of the whole grid."""
    n, steps = 2048, 1000
    r = workloads.sweep_2048(n)[run]
    f = workloads.acoustic_shear(n, n, r.amp)
    with lbm.Grid(n, n, r.tau, r.c2) as g:
        g.init(*f)
        g.step(steps)
        got = g.moments()
    oracle.set_threads(0)
    ref = oracle.simulate(*f, r.tau, r.c2, steps)
    err = _max_err(got, ref)
    tol = _f32_bound(steps, r.amp)
    print(f"2048^2 run {run} (A = {r.amp:.3g}, c2 = {r.c2:.2f}, tau = {r.tau:.3f}): "
          f"max |GPU - oracle| = {err:.2e} (bound {tol:.2e})")
    assert err <= tol


_NEAREST_TOL = {"f32": None, "f16d": 2e-5, "bf16d": 2e-4}


def test_mixed_batch_slice_matches_oracle(lbm):
    """The first 24 grids of the 512-grid batch (sizes 64^2 .. 1024^2, uneven
    aspect, per-grid tau and c^2, sine waves of mode 1-3, amplitude 1e-3) in
    one batch: storages FP32 / FP16-delta / BF16-delta in turn, two 16-bit
    grids with stochastic rounding (small kinds, so their tiles run in the
    general kernel's launch beside the specialised ones), 300 steps with every
    fifth grid stopped at 170.  Every site of every grid against the oracle
    run of its own steps."""
    runs = workloads.batch_grids()[:24]
    kinds = ["f32", "f16d", "bf16d"]
    stochastic = {4, 5}
    steps = 300
    limits = [170 if k % 5 == 0 else steps for k in range(len(runs))]
    grids = []
    for k, r in enumerate(runs):
        g = lbm.Grid(r.nx, r.ny, r.tau, r.c2, kinds[k % 3])
        if k in stochastic:
            g.set_rounding("stochastic")
        g.init(*workloads.sine_wave(r.nx, r.ny, r.amp, r.mode))
        grids.append(g)
    b = lbm.Batch(grids)
    cfg = b.get_config()
    assert cfg["groups"] >= 2 and not cfg["specialised"], cfg
    b.step(steps, limits)
    assert b.sync() == 0
    got = [g.moments() for g in grids]
    b.close()
    for g in grids:
        g.close()
    oracle.set_threads(0)
    worst = {}
    for k, (r, lim, gm) in enumerate(zip(runs, limits, got)):
        ref = oracle.simulate(*workloads.sine_wave(r.nx, r.ny, r.amp, r.mode), r.tau, r.c2, lim)
        kind = kinds[k % 3]
        tol = _f32_bound(lim, r.amp) if kind == "f32" else _NEAREST_TOL[kind]
        if k in stochastic:
            tol *= 2
        err = _max_err(gm, ref)
        name = kind + ("-sr" if k in stochastic else "")
        worst[name] = max(worst.get(name, 0.0), err / tol)
        assert err <= tol, (k, r, name, err, tol)
    print("worst error / bound by kind:", {k: f"{v:.3f}" for k, v in worst.items()})
