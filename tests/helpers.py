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
