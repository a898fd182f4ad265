"""Seeded synthetic inputs for the variable-speed-of-sound D2Q9 runs.

This module only draws numbers: grid sizes, tau and c^2 values, and initial
density / velocity fields.  It holds none of the method's arithmetic, so the
CUDA library, the FP64 oracle and the tests can all take their inputs from it
without sharing any part of the update.

The shapes follow the paper's wave experiments (Section 4: plane sinusoidal
waves on periodic grids, small density amplitudes, rest fluid of unit
density).  The paper runs on no public dataset; every field below is
synthetic.  Recipes (seeds are numpy ``default_rng`` seeds):

* ``sine_wave``        rho = rho0 + A sin(2 pi m x / nx), u = 0 (standing wave)
* ``acoustic_shear``   the standing acoustic wave plus a shear wave
                       u_y = B sin(2 pi x / nx)
* ``progressive_wave`` u = u0 sin(kx), rho = rho0 (1 + (u0/c) sin(kx))
                       (Section 4, waves 1 and 2)
* ``fourier_modes``    rho = 1 + sum of 8 seeded plane waves with integer
                       wave numbers in [-4, 4]^2 \\ {0}, scaled to max
                       |rho - 1| = amp, u = 0
* ``c2_lens``          a per-site c^2 field: c^2 (1 + 0.5 exp(-r^2 / (2 w^2)))
                       around the grid's centre (an acoustic lens)
* ``sweep_2048``       9 runs on 2048^2: c^2 = 0.05 .. 0.45, tau ~ U[0.55, 1.5]
                       (seed 1), amplitudes log-spaced 1e-3 .. 5e-2
* ``batch_grids``      512 grids with log-uniform site counts 64^2 .. 1024^2,
                       aspect 2^U[-2, 2], sides multiples of 8 (seed 4),
                       tau ~ U[0.55, 1.2], c^2 ~ U[0.05, 0.4], mode m in {1,2,3}
* ``serve_trace``      Poisson arrivals (seed 5), log-uniform site counts
                       128^2 .. 2048^2, step counts U{1000 .. 20000}, half
                       FP32 and half FP16-delta storage
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def sine_wave(nx: int, ny: int, amp: float = 1e-3, m: int = 1,
              rho0: float = 1.0):
    """Standing acoustic wave: rho = rho0 + amp sin(2 pi m x / nx), u = 0."""
    x = np.arange(nx, dtype=np.float64)
    rho = np.broadcast_to(rho0 + amp * np.sin(2 * np.pi * m * x / nx),
                          (ny, nx)).copy()
    z = np.zeros((ny, nx))
    return rho, z, z.copy()


def acoustic_shear(nx: int, ny: int, amp: float = 1e-3, shear: float = 1e-3):
    """Standing acoustic wave of amplitude ``amp`` in rho plus a transverse
    shear wave u_y = shear * sin(2 pi x / nx)."""
    rho, ux, uy = sine_wave(nx, ny, amp)
    x = np.arange(nx, dtype=np.float64)
    uy[:] = shear * np.sin(2 * np.pi * x / nx)
    return rho, ux, uy


def progressive_wave(nx: int, ny: int, u0: float, c: float, m: int = 1,
                     rho0: float = 1.0):
    """Right-running wave, Section 4 (waves 1 and 2), read as
    rho = rho0 (1 + (u0 / c) sin(kx)), u_x = u0 sin(kx), u_y = 0."""
    x = np.arange(nx, dtype=np.float64)
    s = np.sin(2 * np.pi * m * x / nx)
    rho = np.broadcast_to(rho0 * (1 + (u0 / c) * s), (ny, nx)).copy()
    ux = np.broadcast_to(u0 * s, (ny, nx)).copy()
    return rho, ux, np.zeros((ny, nx))


def fourier_modes(nx: int, ny: int, amp: float = 1e-3, n_modes: int = 8,
                  seed: int = 3):
    """Random smooth density: 8 plane waves with integer wave numbers
    (kx, ky) in [-4, 4]^2 without (0, 0), phases U[0, 2 pi), weights U[0.5, 1],
    scaled so that max |rho - 1| = amp; u = 0."""
    rng = np.random.default_rng(seed)
    pairs = [(a, b) for a in range(-4, 5) for b in range(-4, 5) if (a, b) != (0, 0)]
    idx = rng.choice(len(pairs), size=n_modes, replace=False)
    phases = rng.uniform(0, 2 * np.pi, n_modes)
    weights = rng.uniform(0.5, 1.0, n_modes)
    x = np.arange(nx, dtype=np.float64)[None, :] / nx
    y = np.arange(ny, dtype=np.float64)[:, None] / ny
    d = np.zeros((ny, nx))
    for j, p in enumerate(idx):
        kx, ky = pairs[p]
        d += weights[j] * np.cos(2 * np.pi * (kx * x + ky * y) + phases[j])
    d *= amp / np.max(np.abs(d))
    z = np.zeros((ny, nx))
    return 1.0 + d, z, z.copy()


def c2_lens(nx: int, ny: int, c2: float, contrast: float = 0.5, width: float = 0.15):
    """A smooth acoustic lens: c^2 raised by `contrast` (relative) in a
    Gaussian bump of relative width `width` at the grid's centre."""
    x = (np.arange(nx, dtype=np.float64)[None, :] + 0.5) / nx - 0.5
    y = (np.arange(ny, dtype=np.float64)[:, None] + 0.5) / ny - 0.5
    return c2 * (1.0 + contrast * np.exp(-(x * x + y * y) / (2 * width * width)))


@dataclass
class Run:
    nx: int
    ny: int
    tau: float
    c2: float
    amp: float
    mode: int = 1


def sweep_2048(n: int = 2048, seed: int = 1):
    """The nine 2048^2 runs: c^2 = 0.05, 0.10, ..., 0.45; tau ~ U[0.55, 1.5];
    acoustic amplitudes log-spaced from 1e-3 to 5e-2."""
    rng = np.random.default_rng(seed)
    taus = rng.uniform(0.55, 1.5, 9)
    amps = np.geomspace(1e-3, 5e-2, 9)
    return [Run(n, n, float(taus[j]), 0.05 * (j + 1), float(amps[j]))
            for j in range(9)]


def batch_grids(count: int = 512, seed: int = 4, lo: int = 64, hi: int = 1024):
    """Uneven grids: sites log-uniform in [lo^2, hi^2], aspect ratio
    2^U[-2, 2], both sides rounded to multiples of 8 (at least 8)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        sites = np.exp(rng.uniform(np.log(lo * lo), np.log(hi * hi)))
        aspect = 2.0 ** rng.uniform(-2, 2)
        nx = max(8, int(round(np.sqrt(sites * aspect) / 8)) * 8)
        ny = max(8, int(round(np.sqrt(sites / aspect) / 8)) * 8)
        tau = float(rng.uniform(0.55, 1.2))
        c2 = float(rng.uniform(0.05, 0.4))
        m = int(rng.integers(1, 4))
        out.append(Run(nx, ny, tau, c2, 1e-3, m))
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    nx: int
    ny: int
    tau: float
    c2: float
    steps: int
    storage: str  # "f32" or "f16d"
    amp: float = 1e-3


def serve_trace(count: int = 2000, rate_hz: float = 200.0, seed: int = 5,
                lo: int = 128, hi: int = 2048, steps_lo: int = 1000,
                steps_hi: int = 20000):
    """Poisson request trace for the serving loop."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, count))
    out = []
    for r in range(count):
        sites = np.exp(rng.uniform(np.log(lo * lo), np.log(hi * hi)))
        aspect = 2.0 ** rng.uniform(-1, 1)
        nx = max(8, int(round(np.sqrt(sites * aspect) / 8)) * 8)
        ny = max(8, int(round(np.sqrt(sites / aspect) / 8)) * 8)
        out.append(Request(r, float(t[r]), nx, ny,
                           float(rng.uniform(0.55, 1.2)),
                           float(rng.uniform(0.05, 0.4)),
                           int(rng.integers(steps_lo, steps_hi + 1)),
                           "f32" if rng.random() < 0.5 else "f16d"))
    return out
