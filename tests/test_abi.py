"""CPU checks of the C ABI library: it builds, loads, exports every function
include/lbm.h declares, and rejects invalid arguments before any device work.
No kernel runs here."""
import ctypes
import os
import re

import pytest

from paper_0707_2437_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_covers_status_codes():
    lib = lbm.load()
    for code, word in [(0, "ok"), (-1, "invalid"), (-2, "memory"), (-3, "CUDA"),
                       (-4, "non-finite"), (-5, "timed out"), (1, "warning")]:
        assert word in lib.lbm_strerror(code).decode()


@pytest.mark.parametrize("args", [
    (0, 8, 0.8, 0.2, 0), (8, 0, 0.8, 0.2, 0), (8, 8, 0.5, 0.2, 0), (8, 8, 0.3, 0.2, 0),
    (8, 8, 0.8, 0.0, 0), (8, 8, 0.8, -0.1, 0), (8, 8, 0.8, 0.2, 3), (8, 8, float("nan"), 0.2, 0),
    (70000, 70000, 0.8, 0.2, 0),
])
def test_create_rejects_invalid_arguments(args):
    lib = lbm.load()
    h = ctypes.c_void_p()
    rc = lib.lbm_create(*args, None, ctypes.byref(h))
    assert rc == -1, (args, rc)
    assert not h.value
    assert "lbm_create" in lib.lbm_last_error().decode()


def test_null_handles_are_rejected():
    lib = lbm.load()
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_init(None, None, None, None, 0) == -1
    assert lib.lbm_destroy(None) == 0
    assert lib.lbm_batch_create(None, 0, None) == -1
    assert lib.lbm_time(None) == -1


def test_bytes_required():
    lib = lbm.load()
    assert lib.lbm_bytes_required(2048, 2048, 0) == 2 * 9 * 2048 * 2048 * 4
    assert lib.lbm_bytes_required(8192, 8192, 1) == 2 * 9 * 8192 * 8192 * 2
    # planes are padded to 64 elements
    assert lib.lbm_bytes_required(3, 3, 0) == 2 * 9 * 64 * 4
    assert lib.lbm_bytes_required(0, 3, 0) == 0


def test_every_handle_call_rejects_null_before_device_work():
    """Every call that takes a grid or batch handle returns LBM_EINVAL for
    NULL, with no CUDA call (this host has no GPU)."""
    lib = lbm.load()
    i = ctypes.c_int()
    d = ctypes.c_double()
    ll = ctypes.c_longlong()
    buf = (ctypes.c_double * 8)()
    grid_calls = [
        lambda: lib.lbm_moments(None, None, None, None, 0),
        lambda: lib.lbm_sums(None, buf),
        lambda: lib.lbm_mode(None, 0, 1, 0, buf),
        lambda: lib.lbm_set_drive(None, 1, 1e-3, 500.0),
        lambda: lib.lbm_set_c2_field(None, None, 0),
        lambda: lib.lbm_sync(None),
        lambda: lib.lbm_set_stream(None, None),
        lambda: lib.lbm_get_state(None, buf, ctypes.byref(ll)),
        lambda: lib.lbm_set_state(None, buf, 0),
        lambda: lib.lbm_set_config(None, 4, 16, 4),
        lambda: lib.lbm_get_config(None, ctypes.byref(i), ctypes.byref(i), ctypes.byref(i)),
        lambda: lib.lbm_set_pipeline(None, 1),
        lambda: lib.lbm_get_pipeline(None, ctypes.byref(i), ctypes.byref(i)),
        lambda: lib.lbm_set_rounding(None, 0),
        lambda: lib.lbm_get_rounding(None, ctypes.byref(i)),
        lambda: lib.lbm_tune(None, None),
        lambda: lib.lbm_set_timing(None, 1),
        lambda: lib.lbm_kernel_ms(None, ctypes.byref(d), ctypes.byref(ll)),
        lambda: lib.lbm_set_persistent(None, 1),
        lambda: lib.lbm_set_persistent(None, 2),
        lambda: lib.lbm_set_gradient(None, 1),
        lambda: lib.lbm_get_gradient(None, ctypes.byref(i)),
    ]
    batch_calls = [
        lambda: lib.lbm_batch_step(None, 1, None),
        lambda: lib.lbm_batch_sync(None),
        lambda: lib.lbm_batch_set_config(None, 16, 0),
        lambda: lib.lbm_batch_tune(None),
        lambda: lib.lbm_batch_get_config(None, ctypes.byref(i), ctypes.byref(i), ctypes.byref(i)),
        lambda: lib.lbm_batch_get_groups(None, ctypes.byref(i)),
        lambda: lib.lbm_batch_get_tiles(None, ctypes.byref(i), ctypes.byref(i)),
        lambda: lib.lbm_batch_set_walk16(None, 0),
        lambda: lib.lbm_batch_get_walk16(None, ctypes.byref(i)),
        lambda: lib.lbm_batch_set_timeout_us(None, 1000),
        lambda: lib.lbm_batch_set_launch(None, 0),
        lambda: lib.lbm_batch_set_schedule(None, 0),
        lambda: lib.lbm_slab_pack(None, buf, 0),
        lambda: lib.lbm_slab_unpack(None, buf, 0),
        lambda: lib.lbm_slab_create(8, 8, 0.8, 0.2, 0, None, None),
        lambda: lib.lbm_batch_get_schedule(None, ctypes.byref(i)),
        lambda: lib.lbm_batch_get_launch(None, ctypes.byref(i), ctypes.byref(i),
                                         ctypes.byref(i)),
    ]
    for k, call in enumerate(grid_calls + batch_calls):
        assert call() == -1, k
    assert lib.lbm_batch_destroy(None) == 0
    assert lib.lbm_state_bytes(None) == 0
    assert lib.lbm_slab_halo_bytes(None) == 0
