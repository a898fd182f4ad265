"""Python binding of liblbm.so (ctypes; argument marshalling only).

Every step of the path runs in the library's CUDA kernels.  This module
converts Python values to the C types of ``include/lbm.h`` and raises
``LbmError`` on a non-zero status.  Arrays may be numpy arrays (host) or
CUDA torch tensors (device pointers are passed through); PyTorch is only used
for device memory and streams.  If the library cannot be built or loaded the
import of the binding fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

STORAGE = {"f32": 0, "f16d": 1, "bf16d": 2}
BYTES_PER_LU = {"f32": 72, "f16d": 36, "bf16d": 36}  # algorithmic bytes per lattice update
FIELD = {"rho": 0, "ux": 1, "uy": 2}
LBM_OK, LBM_WUNSTABLE = 0, 1
LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT = -1, -2, -3, -4, -5

_lib = None
_lock = threading.Lock()


class LbmError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = _lib
        msg = lib.lbm_strerror(status).decode() if lib else str(status)
        detail = lib.lbm_last_error().decode() if lib else ""
        super().__init__(f"{what}: {msg} ({status}) {detail}")
        self.status = status


def load() -> ctypes.CDLL:
    """Builds liblbm.so if it is out of date and loads it."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        vp, dp, i, d, ll = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                            ctypes.c_double, ctypes.c_longlong)
        sz = ctypes.c_size_t
        sig = {
            "lbm_create": ([i, i, d, d, i, vp, ctypes.POINTER(vp)], i),
            "lbm_create_ex": ([i, i, d, d, d, i, vp, ctypes.POINTER(vp)], i),
            "lbm_destroy": ([vp], i),
            "lbm_init": ([vp, vp, vp, vp, i], i),
            "lbm_step": ([vp, ll], i),
            "lbm_moments": ([vp, vp, vp, vp, i], i),
            "lbm_sums": ([vp, dp], i),
            "lbm_mode": ([vp, i, i, i, dp], i),
            "lbm_time": ([vp], ll),
            "lbm_sync": ([vp], i),
            "lbm_set_stream": ([vp, vp], i),
            "lbm_bytes_required": ([i, i, i], sz),
            "lbm_mem_info": ([ctypes.POINTER(sz), ctypes.POINTER(sz)], i),
            "lbm_state_bytes": ([vp], sz),
            "lbm_get_state": ([vp, vp, ctypes.POINTER(ll)], i),
            "lbm_set_state": ([vp, vp, ll], i),
            "lbm_set_config": ([vp, i, i, i], i),
            "lbm_get_config": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "lbm_tune": ([vp, ctypes.c_char_p], i),
            "lbm_set_pipeline": ([vp, i], i),
            "lbm_set_rounding": ([vp, i], i),
            "lbm_set_c2_field": ([vp, vp, i], i),
            "lbm_set_drive": ([vp, i, ctypes.c_double, ctypes.c_double], i),
            "lbm_get_rounding": ([vp, ctypes.POINTER(i)], i),
            "lbm_get_pipeline": ([vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "lbm_set_timing": ([vp, i], i),
            "lbm_set_persistent": ([vp, i], i),
            "lbm_kernel_ms": ([vp, dp, ctypes.POINTER(ll)], i),
            "lbm_batch_create": ([ctypes.POINTER(vp), i, ctypes.POINTER(vp)], i),
            "lbm_batch_destroy": ([vp], i),
            "lbm_batch_step": ([vp, ll, ctypes.POINTER(ll)], i),
            "lbm_batch_sync": ([vp], i),
            "lbm_batch_set_config": ([vp, i, i], i),
            "lbm_batch_tune": ([vp], i),
            "lbm_batch_set_walk16": ([vp, i], i),
            "lbm_batch_get_walk16": ([vp, ctypes.POINTER(i)], i),
            "lbm_batch_get_groups": ([vp, ctypes.POINTER(i)], i),
            "lbm_batch_get_config": ([vp, ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(i)], i),
            "lbm_batch_get_tiles": ([vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
            "lbm_set_gradient": ([vp, i], i),
            "lbm_get_gradient": ([vp, ctypes.POINTER(i)], i),
            "lbm_batch_set_timeout_us": ([vp, ll], i),
            "lbm_batch_set_launch": ([vp, i], i),
            "lbm_batch_set_schedule": ([vp, i], i),
            "lbm_batch_get_schedule": ([vp, ctypes.POINTER(i)], i),
            "lbm_batch_get_launch": ([vp, ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(i)], i),
            "lbm_sums_noalloc": ([vp, i, i, sz, i, d, vp, dp], i),
            "lbm_slab_create": ([i, i, d, d, i, vp, ctypes.POINTER(vp)], i),
            "lbm_slab_halo_bytes": ([vp], sz),
            "lbm_slab_pack": ([vp, vp, i], i),
            "lbm_slab_unpack": ([vp, vp, i], i),
            "lbm_strerror": ([i], ctypes.c_char_p),
            "lbm_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int, what: str) -> int:
    if status < 0:
        raise LbmError(status, what)
    return status


def _ptr(a):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA tensor of
    float64."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a.ctypes.data, 0, a
    import torch  # device memory only
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64:
            raise TypeError("fields must be float64")
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0, a
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data, 0, a


def _stream_handle(stream) -> int:
    """cudaStream_t value of None, an integer handle or a torch.cuda.Stream."""
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def new_stream():
    """A new CUDA stream that does not synchronise with the legacy default
    stream (PyTorch's stream pool creates them non-blocking); pass it, or its
    ``cuda_stream`` handle, as a ``stream`` argument and keep it alive."""
    import torch  # streams only
    return torch.cuda.Stream()


def mem_info():
    lib = load()
    f, t = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib.lbm_mem_info(ctypes.byref(f), ctypes.byref(t)), "lbm_mem_info")
    return f.value, t.value


def bytes_required(nx: int, ny: int, storage: str = "f32") -> int:
    return int(load().lbm_bytes_required(nx, ny, STORAGE[storage]))


def sums_noalloc(f_dev_ptr: int, nx: int, ny: int, plane_stride: int, storage: str = "f32",
                 rho0: float = 1.0, stream=None) -> np.ndarray:
    """Grid totals {mass, momentum_x, momentum_y} of a state buffer already in
    device memory, through lbm_sums_noalloc (no allocation by the library)."""
    lib = load()
    out = np.zeros(3)
    _check(lib.lbm_sums_noalloc(ctypes.c_void_p(int(f_dev_ptr)), nx, ny, plane_stride,
                                STORAGE[storage], rho0,
                                ctypes.c_void_p(_stream_handle(stream)),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "lbm_sums_noalloc")
    return out


class Grid:
    """One periodic grid of the variable-speed-of-sound model (lbm_create)."""

    def __init__(self, nx: int, ny: int, tau: float, c2: float, storage: str = "f32",
                 stream=None, rho0: float = 1.0):
        self.lib = load()
        self.nx, self.ny, self.tau, self.c2 = nx, ny, tau, c2
        self.storage = storage
        self.rho0 = rho0
        self._stream = stream
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(_stream_handle(stream))
        self.status = _check(self.lib.lbm_create_ex(nx, ny, tau, c2, rho0, STORAGE[storage], st,
                                                     ctypes.byref(h)), "lbm_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _check(self.lib.lbm_destroy(self.h), "lbm_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, rho, ux, uy):
        (pr, dr, kr), (pu, du, ku), (pv, dv, kv) = _ptr(rho), _ptr(ux), _ptr(uy)
        if not (dr == du == dv):
            raise ValueError("rho, ux, uy must all be on the host or all on the device")
        for a in (kr, ku, kv):
            if tuple(a.shape) != (self.ny, self.nx):
                raise ValueError(f"field shape {tuple(a.shape)} != {(self.ny, self.nx)}")
        _check(self.lib.lbm_init(self.h, pr, pu, pv, dr), "lbm_init")

    def step(self, n: int = 1):
        _check(self.lib.lbm_step(self.h, int(n)), "lbm_step")

    def moments(self, out=None):
        """(rho, ux, uy) as new numpy arrays, or written into ``out``: three
        float64 arrays of shape (ny, nx), all numpy / CPU tensors (host) or all
        CUDA tensors (device)."""
        if out is not None:
            ptrs = [_ptr(a) for a in out]
            on_dev = {p[1] for p in ptrs}
            if len(on_dev) != 1:
                raise ValueError("outputs must all be on the host or all on the device")
            for p in ptrs:
                if tuple(p[2].shape) != (self.ny, self.nx):
                    raise ValueError("output shape mismatch")
            _check(self.lib.lbm_moments(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                        on_dev.pop()), "lbm_moments")
            return out
        arrs = [np.empty((self.ny, self.nx)) for _ in range(3)]
        _check(self.lib.lbm_moments(self.h, *[a.ctypes.data for a in arrs], 0), "lbm_moments")
        return tuple(arrs)

    def sums(self) -> np.ndarray:
        out = np.zeros(3)
        _check(self.lib.lbm_sums(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "lbm_sums")
        return out

    def mode(self, field: str = "rho", kx: int = 1, ky: int = 0) -> np.ndarray:
        out = np.zeros(2)
        _check(self.lib.lbm_mode(self.h, FIELD[field], kx, ky,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "lbm_mode")
        return out

    @property
    def t(self) -> int:
        return int(self.lib.lbm_time(self.h))

    def sync(self):
        _check(self.lib.lbm_sync(self.h), "lbm_sync")

    def set_stream(self, stream):
        """Moves the grid to `stream` (None: the legacy default stream); work
        queued later runs there, after the work already queued."""
        _check(self.lib.lbm_set_stream(self.h, ctypes.c_void_p(_stream_handle(stream))),
               "lbm_set_stream")
        self._stream = stream

    def get_state(self):
        n = int(self.lib.lbm_state_bytes(self.h))
        buf = np.empty(n, dtype=np.uint8)
        t = ctypes.c_longlong()
        _check(self.lib.lbm_get_state(self.h, buf.ctypes.data, ctypes.byref(t)), "lbm_get_state")
        return buf, t.value

    def set_state(self, buf: np.ndarray, t: int):
        buf = np.ascontiguousarray(buf)
        if buf.nbytes != int(self.lib.lbm_state_bytes(self.h)):
            raise ValueError("state size mismatch")
        _check(self.lib.lbm_set_state(self.h, buf.ctypes.data, int(t)), "lbm_set_state")

    def set_config(self, vec: int, rows: int, warps: int):
        _check(self.lib.lbm_set_config(self.h, vec, rows, warps), "lbm_set_config")

    def get_config(self):
        v, r, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.lbm_get_config(self.h, ctypes.byref(v), ctypes.byref(r), ctypes.byref(w)),
               "lbm_get_config")
        return v.value, r.value, w.value

    def set_c2_field(self, c2):
        """Per-site c_e^2 ([ny, nx] float64, host or CUDA), or None for the
        grid's uniform c^2."""
        if c2 is None:
            _check(self.lib.lbm_set_c2_field(self.h, None, 0), "lbm_set_c2_field")
            return
        p, dev, keep = _ptr(c2)
        if tuple(keep.shape) != (self.ny, self.nx):
            raise ValueError("c2 field shape mismatch")
        _check(self.lib.lbm_set_c2_field(self.h, p, dev), "lbm_set_c2_field")

    def set_drive(self, amplitude: float | None, period: float = 500.0):
        """Driven channel in x (Section 4, the Fig. 1 runs): after each step
        column 0 holds the equilibrium at rho = 1 + amplitude sin(2 pi t /
        period), u = 0, and columns nx-2, nx-1 the equilibrium at rho = 1,
        u = 0.  None returns to a periodic grid."""
        if amplitude is None:
            _check(self.lib.lbm_set_drive(self.h, 0, 0.0, 0.0), "lbm_set_drive")
        else:
            _check(self.lib.lbm_set_drive(self.h, 1, float(amplitude), float(period)),
                   "lbm_set_drive")

    def set_rounding(self, mode: str):
        """'nearest' or 'stochastic' (16-bit storage only)."""
        _check(self.lib.lbm_set_rounding(self.h, {"nearest": 0, "stochastic": 1}[mode]),
               "lbm_set_rounding")

    def set_gradient(self, mode: str):
        """'central' (the default, Section 4's scheme) or 'forward' (the
        forward difference, for its instability; FP32 without a c2 field)."""
        _check(self.lib.lbm_set_gradient(self.h, {"central": 0, "forward": 1}[mode]),
               "lbm_set_gradient")

    def get_gradient(self) -> str:
        m = ctypes.c_int()
        _check(self.lib.lbm_get_gradient(self.h, ctypes.byref(m)), "lbm_get_gradient")
        return ["central", "forward"][m.value]

    def get_rounding(self) -> str:
        m = ctypes.c_int()
        _check(self.lib.lbm_get_rounding(self.h, ctypes.byref(m)), "lbm_get_rounding")
        return ["nearest", "stochastic"][m.value]

    def set_pipeline(self, stages: int):
        _check(self.lib.lbm_set_pipeline(self.h, stages), "lbm_set_pipeline")

    def get_pipeline(self):
        st, act = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.lbm_get_pipeline(self.h, ctypes.byref(st), ctypes.byref(act)),
               "lbm_get_pipeline")
        return st.value, bool(act.value)

    def tune(self, cache_path: str | None = None):
        _check(self.lib.lbm_tune(self.h, cache_path.encode() if cache_path else None), "lbm_tune")
        return self.get_config() + (self.get_pipeline()[0],)

    def set_persistent(self, on):
        """True (long calls run one persistent launch), False (never), or
        'auto' (the default: persistent for large 16-bit grids only)."""
        mode = 2 if on == "auto" else (1 if on else 0)
        _check(self.lib.lbm_set_persistent(self.h, mode), "lbm_set_persistent")

    def set_timing(self, on: bool):
        _check(self.lib.lbm_set_timing(self.h, 1 if on else 0), "lbm_set_timing")

    def kernel_ms(self):
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _check(self.lib.lbm_kernel_ms(self.h, ctypes.byref(ms), ctypes.byref(n)), "lbm_kernel_ms")
        return ms.value, n.value


class Slab(Grid):
    """The slab of a grid split along y that one rank owns (lbm_slab_create):
    `ny_local` own rows between two ghost rows on each side; the local buffer
    (fields of init / moments) is [ny_local + 4][nx].  step() takes one step;
    pack / unpack move the halo rows through device buffers."""

    GHOST = 2

    def __init__(self, nx: int, ny_local: int, tau: float, c2: float, storage: str = "f32",
                 stream=None):
        self.lib = load()
        self.nx, self.ny, self.tau, self.c2 = nx, ny_local + 2 * self.GHOST, tau, c2
        self.ny_local = ny_local
        self.storage = storage
        self.rho0 = 1.0
        self._stream = stream
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(_stream_handle(stream))
        self.status = _check(self.lib.lbm_slab_create(nx, ny_local, tau, c2, STORAGE[storage],
                                                       st, ctypes.byref(h)), "lbm_slab_create")
        self.h = h

    @property
    def halo_bytes(self) -> int:
        return int(self.lib.lbm_slab_halo_bytes(self.h))

    def pack(self, side: int, out):
        """Own rows next to `side` (0: the two lowest, 1: the two highest) into
        the device buffer `out` (a CUDA tensor of halo_bytes bytes)."""
        _check(self.lib.lbm_slab_pack(self.h, ctypes.c_void_p(out.data_ptr()), side),
               "lbm_slab_pack")

    def unpack(self, side: int, src):
        """The device buffer `src` into the ghost rows of `side` (0: below,
        1: above)."""
        _check(self.lib.lbm_slab_unpack(self.h, ctypes.c_void_p(src.data_ptr()), side),
               "lbm_slab_unpack")


WALK16 = {"auto": 0, "v8": 1, "v4": 2, "v4pf2": 3}
WALK16_NAMES = {v: k for k, v in WALK16.items()}
LAUNCH = {"auto": 0, "graph": 1, "direct": 2}
SCHEDULE = {"lockstep": 0, "flow": 1}
SCHEDULE_NAMES = {v: k for k, v in SCHEDULE.items()}
LAUNCH_NAMES = {v: k for k, v in LAUNCH.items()}


class Batch:
    """Many grids advanced together by one persistent launch (lbm_batch_*)."""

    def __init__(self, grids):
        self.lib = load()
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        b = ctypes.c_void_p()
        _check(self.lib.lbm_batch_create(arr, len(self.grids), ctypes.byref(b)),
               "lbm_batch_create")
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            _check(self.lib.lbm_batch_destroy(self.b), "lbm_batch_destroy")
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int, limits=None):
        if limits is None:
            _check(self.lib.lbm_batch_step(self.b, int(n), None), "lbm_batch_step")
        else:
            lim = (ctypes.c_longlong * len(self.grids))(*[int(x) for x in limits])
            _check(self.lib.lbm_batch_step(self.b, int(n), lim), "lbm_batch_step")

    def sync(self) -> int:
        return _check(self.lib.lbm_batch_sync(self.b), "lbm_batch_sync")

    def set_config(self, rows: int, blocks_per_sm: int):
        _check(self.lib.lbm_batch_set_config(self.b, rows, blocks_per_sm), "lbm_batch_set_config")

    def tune(self):
        _check(self.lib.lbm_batch_tune(self.b), "lbm_batch_tune")
        return self.get_config()

    def get_config(self):
        r, b, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.lbm_batch_get_config(self.b, ctypes.byref(r), ctypes.byref(b),
                                             ctypes.byref(sp)), "lbm_batch_get_config")
        wk = ctypes.c_int()
        _check(self.lib.lbm_batch_get_walk16(self.b, ctypes.byref(wk)), "lbm_batch_get_walk16")
        ng = ctypes.c_int()
        _check(self.lib.lbm_batch_get_groups(self.b, ctypes.byref(ng)), "lbm_batch_get_groups")
        nt, npair = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.lbm_batch_get_tiles(self.b, ctypes.byref(nt), ctypes.byref(npair)),
               "lbm_batch_get_tiles")
        return {"rows": r.value, "blocks_per_sm": b.value, "specialised": bool(sp.value),
                "walk16": WALK16_NAMES[wk.value], "groups": ng.value, "tiles": nt.value,
                "paired_tiles": npair.value}

    def set_walk16(self, walk: str):
        """Walk of the batch's 16-bit grids: 'auto' (the default, 'v8'), 'v8'
        (8 sites per lane), 'v4' (4 per lane, one row prefetched) or 'v4pf2'
        (two rows)."""
        _check(self.lib.lbm_batch_set_walk16(self.b, WALK16[walk]), "lbm_batch_set_walk16")

    def set_timeout_us(self, us: int):
        _check(self.lib.lbm_batch_set_timeout_us(self.b, int(us)), "lbm_batch_set_timeout_us")

    def set_schedule(self, schedule: str):
        """'lockstep' (the default: a grid-wide barrier between time steps) or
        'flow' (each grid advances on its own, per-tile progress)."""
        _check(self.lib.lbm_batch_set_schedule(self.b, SCHEDULE[schedule]),
               "lbm_batch_set_schedule")

    def get_schedule(self) -> str:
        v = ctypes.c_int()
        _check(self.lib.lbm_batch_get_schedule(self.b, ctypes.byref(v)), "lbm_batch_get_schedule")
        return SCHEDULE_NAMES[v.value]

    def set_launch(self, mode: str):
        """'auto' (graph replay, direct launches if capture fails), 'graph'
        (capture failure is an error) or 'direct'."""
        _check(self.lib.lbm_batch_set_launch(self.b, LAUNCH[mode]), "lbm_batch_set_launch")

    def get_launch(self):
        """{'mode', 'last' ('graph', 'direct' or None before the first step
        call), 'capture_failed'}."""
        m, last, cf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.lbm_batch_get_launch(self.b, ctypes.byref(m), ctypes.byref(last),
                                             ctypes.byref(cf)), "lbm_batch_get_launch")
        return {"mode": LAUNCH_NAMES[m.value],
                "last": {0: None, 1: "graph", 2: "direct"}[last.value],
                "capture_failed": bool(cf.value)}
