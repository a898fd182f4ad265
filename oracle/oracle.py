"""Python access to the FP64 CPU oracle in ``lbm_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, the bench's CPU-baseline leg and the
smoke check use this module; the product library never does.  It shares no
code with the CUDA path.

The oracle computes the variable-speed-of-sound D2Q9 update of Buick &
Cosgrove, Section 3, Eq. 5 (nbm), in double precision:

    f_i(x+e_i, t+1) = f_i - (f_i - fbar_i)/tau + 3 w_i alpha grad(rho).e_i

with the equilibrium of Section 2, Eq. 2, the moments of Eq. 3 and the weights
and link vectors of Section 2.  The sound speed is c_e = sqrt(c_1^2 - alpha),
Section 3, Eq. 8 (cef), with c_1^2 = 1/3 for this lattice: the paper fixes that
value through alpha = 1/3 giving c_e = 0 and alpha = -2/3 giving c_e = 1
(Section 4), and alpha = 0.2933 giving c_e = 0.2 (Section 4, wave 1).

Array layout: distributions ``f`` are float64 ``[9, ny, nx]`` (the state
f_i(x, t) before collision, already streamed); fields are ``[ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

C1_SQ = 1.0 / 3.0  # squared lattice sound speed of D2Q9 (Section 4 values)

# Link vectors and weights, Section 2 (listed for tests that need them).
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

GRAD = {"central": 0, "forward": 1}


def build(force: bool = False) -> str:
    """Compiles ``lbm_oracle.c`` into ``_build/liblbm_oracle.so`` (gcc, -O3,
    OpenMP).  Returns the library path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_equilibrium.argtypes = [ctypes.c_double] * 3 + [dp]
        lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.oracle_moments.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int,
                                   ctypes.c_long, dp]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run_field.argtypes = [ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, dp, ctypes.c_int,
                                         ctypes.c_long, dp]
        lib.oracle_run_field.restype = ctypes.c_int
        lib.oracle_sums.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_run_driven.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_long, ctypes.c_long,
                                          ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_run_driven.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def alpha_from_c2(c2: float) -> float:
    """alpha = c_1^2 - c_e^2, from Section 3, Eq. 8 (cef) with c_1^2 = 1/3."""
    return C1_SQ - c2


def set_threads(n: int) -> int:
    """Sets the OpenMP thread count of the oracle; returns the count used."""
    return _load().oracle_set_threads(int(n))


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    """fbar_i(rho, u) of Section 2, Eq. 2, for i = 0..8."""
    out = np.zeros(9)
    _load().oracle_equilibrium(rho, ux, uy, _ptr(out))
    return out


def init(rho: np.ndarray, ux: np.ndarray, uy: np.ndarray) -> np.ndarray:
    """Initial state f_i = fbar_i(rho, u) at every site; returns [9, ny, nx]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ux = np.ascontiguousarray(ux, dtype=np.float64)
    uy = np.ascontiguousarray(uy, dtype=np.float64)
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    _load().oracle_init(nx, ny, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(f))
    return f


def moments(f: np.ndarray):
    """(rho, ux, uy) of the state f, Section 2, Eq. 3."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    rho, ux, uy = (np.zeros((ny, nx)) for _ in range(3))
    _load().oracle_moments(nx, ny, _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def run(f: np.ndarray, tau: float, alpha, steps: int,
        grad: str = "central") -> np.ndarray:
    """Advances the state f by ``steps`` steps of Eq. 5 in place and returns it.
    ``alpha`` is a number, or a [ny, nx] field (spatially varying alpha)."""
    assert f.dtype == np.float64 and f.flags["C_CONTIGUOUS"]
    _, ny, nx = f.shape
    lib = _load()
    if np.ndim(alpha) == 0:
        rc = lib.oracle_run(nx, ny, float(tau), float(alpha), GRAD[grad],
                            int(steps), _ptr(f))
    else:
        al = np.ascontiguousarray(alpha, dtype=np.float64)
        assert al.shape == (ny, nx)
        rc = lib.oracle_run_field(nx, ny, float(tau), _ptr(al), GRAD[grad],
                                  int(steps), _ptr(f))
    if rc != 0:
        raise MemoryError("oracle_run: allocation failed")
    return f


def run_driven(f: np.ndarray, tau: float, alpha: float, t0: int, steps: int, amp: float,
               period: float) -> np.ndarray:
    """Driven channel of Section 4 (the runs of Fig. 1), in place.  After each
    collision the post-collision distributions of column 0 become the
    equilibrium at rho = 1 + amp sin(2 pi t / period), u = 0, and those of
    columns nx-2 and nx-1 the equilibrium at rho = 1, u = 0 (the reading taken
    where the paper names the boundary values but no scheme); periodic in y.
    Steps t = t0 .. t0+steps-1; needs nx >= 4."""
    assert f.dtype == np.float64 and f.flags["C_CONTIGUOUS"]
    _, ny, nx = f.shape
    rc = _load().oracle_run_driven(nx, ny, float(tau), float(alpha), int(t0), int(steps),
                                   float(amp), float(period), _ptr(f))
    if rc == -2:
        raise ValueError("oracle_run_driven: needs nx >= 4")
    if rc != 0:
        raise MemoryError("oracle_run_driven: allocation failed")
    return f


def sums(f: np.ndarray) -> np.ndarray:
    """[mass, momentum_x, momentum_y] summed over the grid."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    out = np.zeros(3)
    _load().oracle_sums(nx, ny, _ptr(f), _ptr(out))
    return out


def simulate(rho0, ux0, uy0, tau: float, c2: float, steps: int,
             grad: str = "central"):
    """Equilibrium init from (rho0, ux0, uy0), ``steps`` steps with
    alpha = 1/3 - c2, and the moments of the final state."""
    f = init(rho0, ux0, uy0)
    run(f, tau, alpha_from_c2(c2), steps, grad)
    return moments(f)
