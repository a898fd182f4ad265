"""Exact-rational brute force of the variable-speed-of-sound D2Q9 update.

TEST INFRASTRUCTURE ONLY: pins the FP64 oracle on tiny grids.

Everything is a ``fractions.Fraction``, so the result is the exact value of
Section 3, Eq. 5 (nbm) for rational inputs.  It is written independently of
``lbm_oracle.c`` and deliberately in the other streaming form: here each site
*pulls* f_i(x, t+1) = f*_i(x - e_i, t) (the same update as pushing f*_i(x, t)
to x + e_i).  Central differences for grad(rho) (Section 4), periodic wrap,
equilibrium of Section 2, Eq. 2, moments of Eq. 3.
"""
from __future__ import annotations

from fractions import Fraction as Q

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
     (1, 1), (-1, 1), (-1, -1), (1, -1)]
WQ = [Q(4, 9)] + [Q(1, 9)] * 4 + [Q(1, 36)] * 4


def feq(rho, ux, uy):
    usq = ux * ux + uy * uy
    out = []
    for (ex, ey), w in zip(E, WQ):
        eu = ex * ux + ey * uy
        out.append(w * rho * (1 + 3 * eu + Q(9, 2) * eu * eu - Q(3, 2) * usq))
    return out


def init(rho, ux, uy):
    """rho, ux, uy: lists of rows of Fractions.  Returns f[y][x][i]."""
    ny, nx = len(rho), len(rho[0])
    return [[feq(rho[y][x], ux[y][x], uy[y][x]) for x in range(nx)]
            for y in range(ny)]


def moments(f):
    ny, nx = len(f), len(f[0])
    rho = [[sum(f[y][x]) for x in range(nx)] for y in range(ny)]
    ux = [[sum(f[y][x][i] * E[i][0] for i in range(9)) / rho[y][x]
           for x in range(nx)] for y in range(ny)]
    uy = [[sum(f[y][x][i] * E[i][1] for i in range(9)) / rho[y][x]
           for x in range(nx)] for y in range(ny)]
    return rho, ux, uy


def step(f, tau, alpha):
    """One step of Eq. 5.  ``alpha`` is a Fraction, or rows of Fractions: a
    per-site alpha (the spatially varying sound speed of Section 5), used in
    the force at the site where the collision happens."""
    ny, nx = len(f), len(f[0])
    rho, ux, uy = moments(f)
    per_site = isinstance(alpha, list)
    post = [[None] * nx for _ in range(ny)]
    for y in range(ny):
        for x in range(nx):
            gx = (rho[y][(x + 1) % nx] - rho[y][(x - 1) % nx]) / 2
            gy = (rho[(y + 1) % ny][x] - rho[(y - 1) % ny][x]) / 2
            eq = feq(rho[y][x], ux[y][x], uy[y][x])
            a = alpha[y][x] if per_site else alpha
            post[y][x] = [f[y][x][i] - (f[y][x][i] - eq[i]) / tau
                          + 3 * WQ[i] * a * (gx * E[i][0] + gy * E[i][1])
                          for i in range(9)]
    return [[[post[(y - E[i][1]) % ny][(x - E[i][0]) % nx][i] for i in range(9)]
             for x in range(nx)] for y in range(ny)]


def run(f, tau, alpha, steps):
    for _ in range(steps):
        f = step(f, tau, alpha)
    return f
