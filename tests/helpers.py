"""Measurement helpers shared by the tests (plain numpy / scipy, FP64)."""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares


def mode_sin_cos(field: np.ndarray, m: int = 1):
    """Projection of a [ny, nx] field on sin and cos of 2 pi m x / nx,
    averaged over y: returns (a_sin, a_cos) with field ~ a_sin sin + a_cos cos."""
    ny, nx = field.shape
    x = np.arange(nx)
    s = np.sin(2 * np.pi * m * x / nx)
    c = np.cos(2 * np.pi * m * x / nx)
    prof = field.mean(axis=0)
    return 2.0 * prof @ s / nx, 2.0 * prof @ c / nx


def fit_damped_cos(t: np.ndarray, a: np.ndarray, omega0: float, gamma0: float):
    """Least-squares fit a(t) = A exp(-gamma t) cos(omega t + phi).
    Returns (omega, gamma, A, phi)."""
    def resid(p):
        A, g, w, ph = p
        return A * np.exp(-g * t) * np.cos(w * t + ph) - a

    amp0 = np.max(np.abs(a))
    r = least_squares(resid, [amp0, gamma0, omega0, 0.0], xtol=1e-15,
                      ftol=1e-15, gtol=1e-15, max_nfev=20000)
    A, g, w, ph = r.x
    return w, g, A, ph


def fit_decay(t: np.ndarray, a: np.ndarray):
    """Least-squares slope of ln|a| against t: returns the damping rate."""
    return -np.polyfit(t, np.log(np.abs(a)), 1)[0]


def harmonic_amplitudes(profile: np.ndarray, n: int = 4):
    """|FFT| amplitudes a_1..a_n of a periodic 1-D profile."""
    F = np.fft.rfft(profile)
    return 2.0 * np.abs(F[1:n + 1]) / len(profile)


def phasor(t: np.ndarray, s: np.ndarray, omega: float) -> complex:
    """Least-squares complex amplitude Z of s(t) ~ Re(Z exp(i omega t)) + c."""
    M = np.stack([np.cos(omega * t), -np.sin(omega * t), np.ones_like(t)], axis=1)
    (a, b, _), *_ = np.linalg.lstsq(M, s, rcond=None)
    return complex(a, b)


def driven_plan(ce: float, period: float = 500.0):
    """Probe layout for the driven-channel sound-speed runs (Section 4, Fig. 1):
    probes at x1 and x1 + D with the travel time D / c_e about 0.4 period (so
    the phase delay is unambiguous for speeds above 0.4 c_e), a window of two
    whole periods starting two periods after the front passed the far probe,
    sampled every ``every`` steps.  Returns (x1, D, t_start, t_end, every)."""
    x1 = max(10, int(round(0.3 * period * ce)))
    D = max(8, int(round(0.4 * period * ce)))
    t_start = int(np.ceil((x1 + D) / ce + 2 * period))
    return x1, D, t_start, t_start + int(2 * period), 10


def driven_estimates(t, rho1, rho2, u1, D: int, omega: float):
    """The two sound-speed estimates of Section 4 from probe series:
    time of flight D / delay, with the delay the phase lag of the density at
    the far probe over omega; and the plane-wave relation u / c_e =
    (rho - rho0) / rho0 (rho0 = 1) at the near probe, c = |U| / |R| of the
    fundamental.  Returns (c_tof, c_imp)."""
    t = np.asarray(t, float)
    z1 = phasor(t, np.asarray(rho1) - 1.0, omega)
    z2 = phasor(t, np.asarray(rho2) - 1.0, omega)
    zu = phasor(t, np.asarray(u1), omega)
    lag = (-np.angle(z2 / z1)) % (2 * np.pi)
    c_tof = D * omega / lag
    c_imp = abs(zu) / abs(z1)
    return float(c_tof), float(c_imp)


def oracle_cone_window(fields, tau: float, alpha: float, steps: int, y0: int, x0: int, h: int,
                       w: int, crop_every: int = 100):
    """Exact oracle moments after ``steps`` steps on the window [y0, y0+h) x
    [x0, x0+w) of a large periodic grid, computed from the window's dependency
    cone only.  The central-difference step of Eq. 5 reaches 2 sites per step
    (streaming 1, the gradient 1 more), so a periodic oracle run on the window
    grown by 2 (steps - t) + 2 on each side is exact on the target window at
    step ``steps``; the state is re-cropped every ``crop_every`` steps as the
    cone narrows.  ``fields`` = (rho, ux, uy) of the whole grid, [ny, nx]."""
    from oracle import oracle

    ny, nx = fields[0].shape
    m = 2 * steps + 2
    ys = np.arange(y0 - m, y0 + h + m) % ny
    xs = np.arange(x0 - m, x0 + w + m) % nx
    f = oracle.init(*(np.ascontiguousarray(a[np.ix_(ys, xs)]) for a in fields))
    t = 0
    while t < steps:
        n = min(crop_every, steps - t)
        oracle.run(f, tau, alpha, n)
        t += n
        cut = m - (2 * (steps - t) + 2)
        if cut > 0:
            f = np.ascontiguousarray(f[:, cut:f.shape[1] - cut, cut:f.shape[2] - cut])
            m -= cut
    r, u, v = oracle.moments(f)
    sl = (slice(m, m + h), slice(m, m + w))
    return r[sl], u[sl], v[sl]


def linear_mode_prediction(z0: complex, kx: float, ky: float, tau: float, alpha: float,
                           steps: int, zux: complex = 0j, zuy: complex = 0j):
    """Complex amplitudes (rho, u_x, u_y) after ``steps`` steps of a mode that
    starts as the equilibrium at rho = 1 + Re(z0 exp(i k.x)),
    u = Re((zux, zuy) exp(i k.x)), by the linearised update M(k) (wavevector
    in radians per site; first order in the amplitudes, rho0 = 1).  With
    zux = zuy = 0 returns the density amplitude alone."""
    from oracle import linear

    M = linear.update_matrix(kx, ky, tau, alpha)
    a0 = linear.W * (z0 + 3.0 * (linear.EX * zux + linear.EY * zuy))
    a = np.linalg.matrix_power(M, steps) @ a0
    if zux == 0 and zuy == 0:
        return complex(a.sum())
    return complex(a.sum()), complex(a @ linear.EX), complex(a @ linear.EY)


def low_modes(field: np.ndarray, kmax: int = 4):
    """(2/N) sum field exp(-i k.x) for integer wave numbers |kx|, |ky| <= kmax,
    as a [2 kmax + 1, 2 kmax + 1] array indexed [ky + kmax, kx + kmax]."""
    ny, nx = field.shape
    ks = np.arange(-kmax, kmax + 1)
    ex = np.exp(-2j * np.pi * np.outer(ks, np.arange(nx)) / nx)
    ey = np.exp(-2j * np.pi * np.outer(ks, np.arange(ny)) / ny)
    return 2.0 * (ey @ (field @ ex.T)) / (nx * ny)
