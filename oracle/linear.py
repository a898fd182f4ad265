"""Linear (small-amplitude) analysis of the variable-speed-of-sound D2Q9 update.

TEST INFRASTRUCTURE ONLY (used by the tests to pin the oracle and to state the
exact discrete sound speed and damping a simulation should show).

A perturbation f_i = w_i rho0 + a_i exp(i k.x) about rest (rho0, u = 0) of
Section 3, Eq. 5 (nbm), evolves per step as a -> M(k) a with

    M(k) = S(k) [ (1 - 1/tau) I + (1/tau) E + F(k) ]

  * E_ij = w_i (1 + 3 e_i.e_j): the equilibrium of Section 2, Eq. 2, kept to
    first order in the perturbation (rho0 u = sum_j a_j e_j to this order, so
    rho0 drops out);
  * F_ij = 3 w_i alpha (e_i.g(k)): the force of Eq. 5, with grad(rho) of a mode
    equal to g(k) times its density amplitude sum_j a_j; central differences
    (Section 4) give g = (i sin kx, i sin ky), the forward difference gives
    g = (exp(i kx) - 1, exp(i ky) - 1);
  * S_ii = exp(-i k.e_i): streaming along e_i (left-hand side of Eq. 5).

An eigenvalue lambda of M gives one mode's per-step growth: damping
Gamma = -ln|lambda| and angular frequency omega = |arg lambda|.  For small k
the three hydrodynamic modes have omega = c_e |k| with c_e^2 = 1/3 - alpha
(Section 3, Eq. 8) and shear damping nu |k|^2 with nu = (2 tau - 1)/6
(Section 3, Eq. 7).
"""
from __future__ import annotations

import numpy as np

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def update_matrix(kx: float, ky: float, tau: float, alpha: float,
                  grad: str = "central") -> np.ndarray:
    """The 9x9 complex matrix M(k) described in the module docstring."""
    ee = np.outer(EX, EX) + np.outer(EY, EY)
    E = W[:, None] * (1.0 + 3.0 * ee)
    if grad == "central":
        gx, gy = 1j * np.sin(kx), 1j * np.sin(ky)
    elif grad == "forward":
        gx, gy = np.exp(1j * kx) - 1.0, np.exp(1j * ky) - 1.0
    else:
        raise ValueError(grad)
    F = (3.0 * W * alpha * (EX * gx + EY * gy))[:, None] * np.ones((1, 9))
    C = (1.0 - 1.0 / tau) * np.eye(9) + E / tau + F
    S = np.diag(np.exp(-1j * (kx * EX + ky * EY)))
    return S @ C


def eigen(kx: float, ky: float, tau: float, alpha: float,
          grad: str = "central"):
    """Eigenvalues and eigenvectors of M(k) (numpy.linalg.eig)."""
    return np.linalg.eig(update_matrix(kx, ky, tau, alpha, grad))


def hydro_modes(kx: float, ky: float, tau: float, alpha: float,
                grad: str = "central"):
    """The acoustic pair and the shear mode at small k.

    Returns a dict with ``omega`` (angular frequency per step of the acoustic
    modes), ``gamma_sound`` (their damping per step) and ``gamma_shear`` (the
    damping per step of the non-oscillating shear mode).  Modes are told apart
    by the density content of their eigenvectors: the acoustic modes carry
    density, the shear mode carries transverse momentum only.
    """
    lam, vec = eigen(kx, ky, tau, alpha, grad)
    k = np.hypot(kx, ky)
    # The three modes closest to |lambda| = 1 are the hydrodynamic ones.
    order = np.argsort(-np.abs(lam))
    hyd = order[:3]
    dens = np.abs(vec[:, hyd].sum(axis=0)) / np.linalg.norm(vec[:, hyd], axis=0)
    shear = hyd[np.argmin(dens)]
    sound = [m for m in hyd if m != shear]
    om = np.abs(np.angle(lam[sound]))
    gs = -np.log(np.abs(lam[sound]))
    return {
        "omega": float(om.mean()),
        "c": float(om.mean() / k),
        "gamma_sound": float(gs.mean()),
        "gamma_shear": float(-np.log(np.abs(lam[shear]))),
        "lambda": lam,
    }


def spectral_radius(kx: float, ky: float, tau: float, alpha: float,
                    grad: str = "central") -> float:
    """max |lambda| of M(k); above 1 the mode grows (linear instability)."""
    return float(np.max(np.abs(np.linalg.eigvals(
        update_matrix(kx, ky, tau, alpha, grad)))))


def max_growth(n: int, tau: float, alpha: float, grad: str = "central") -> float:
    """max over all wavevectors of an n x n periodic grid of the spectral
    radius of M(k)."""
    ks = 2 * np.pi * np.arange(n) / n
    return max(spectral_radius(kx, ky, tau, alpha, grad)
               for kx in ks for ky in ks)


def driven_wave(omega: float, tau: float, alpha: float, grad: str = "central"):
    """The wave a boundary driven at angular frequency ``omega`` (per step)
    sends along +x, as in the sound-speed runs of Section 4: the complex
    wavenumber k at which M(k, 0) has the eigenvalue exp(-i omega), so that
    a_i exp(i (k x - omega t)) is a mode (Im k > 0: spatial decay).

    Returns a dict with ``k``, ``c_phase`` = omega / Re k (the speed a
    time-of-flight measurement sees), ``impedance`` = U / R (complex: the
    x-velocity over the density amplitude of the eigenvector, U = sum a_i
    e_ix, R = sum a_i; the plane-wave relation of Section 4 gives
    U / R = c_e at rho0 = 1) and ``decay`` = Im k per lattice unit.
    Solved by the secant method on k from omega / sqrt(1/3 - alpha)."""
    target = np.exp(-1j * omega)

    def g(k):
        lam = np.linalg.eigvals(update_matrix(k, 0.0, tau, alpha, grad))
        return lam[np.argmin(np.abs(lam - target))] - target

    k0 = omega / np.sqrt(1.0 / 3.0 - alpha) + 0j
    k1 = k0 * (1 + 1e-3)
    g0, g1 = g(k0), g(k1)
    for _ in range(100):
        if g1 == g0:
            break
        k2 = k1 - g1 * (k1 - k0) / (g1 - g0)
        k0, g0, k1 = k1, g1, k2
        g1 = g(k1)
        if abs(g1) < 1e-14:
            break
    lam, vec = np.linalg.eig(update_matrix(k1, 0.0, tau, alpha, grad))
    v = vec[:, np.argmin(np.abs(lam - target))]
    R, U = v.sum(), (v * EX).sum()
    return {"k": complex(k1), "c_phase": float(omega / k1.real),
            "impedance": complex(U / R), "decay": float(k1.imag),
            "residual": float(abs(g1))}
