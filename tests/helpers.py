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
