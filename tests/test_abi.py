"""Host-side checks of the C ABI: the library loads, exports every function
include/da.h declares, validates its arguments, and has no CPU fallback."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?\s*(da_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libda():
    import __graft_entry__
    from paper_1806_08815_gb300 import build, binding
    build.build()
    return binding.lib()


# The boundary the library is built around: instance contexts and the anneal
# (Algorithm 2), PTDA (Sec. II, Algorithm 4), the request loop, the batched and
# plain forms, the allocation-free anneal, exact energies and the diagnostics
# the tests use.
REQUIRED = ("da_create", "da_destroy", "da_anneal", "da_anneal_async", "da_pt", "da_pt_adaptive",
            "da_last_error", "da_energy", "da_field_recompute",
            "da_server_create", "da_submit", "da_poll", "da_cancel", "da_req_free", "da_server_stats",
            "da_server_destroy",
            "da_batch_anneal", "da_anneal_plain", "da_anneal_static", "da_static_pitch",
            "da_quantize", "da_move_energy_percentiles", "da_tts_bootstrap", "da_percentiles",
            "da_diag_fail_alloc", "da_diag_live_allocations", "da_anneal_segment", "da_tune_shape",
            "da_batch_describe", "da_batch_force", "da_server_resident", "da_diag_read_bandwidth")


def test_header_declares_the_boundary():
    names = declared_functions()
    missing = [r for r in REQUIRED if r not in names]
    assert not missing, missing


def test_library_exports_every_declared_symbol(libda):
    missing = [n for n in declared_functions() if not hasattr(libda, n)]
    assert not missing, missing


def test_argument_validation_without_device(libda):
    from paper_1806_08815_gb300 import binding as b
    h = ctypes.c_void_p()
    Q = np.zeros((4, 4), np.int32)
    assert libda.da_create(Q.ctypes.data_as(ctypes.c_void_p), 0, 0, ctypes.byref(h)) == 1      # N = 0
    assert libda.da_create(Q.ctypes.data_as(ctypes.c_void_p), 9000, 0, ctypes.byref(h)) == 1   # N > 8192
    assert libda.da_create(Q.ctypes.data_as(ctypes.c_void_p), 4, 7, ctypes.byref(h)) == 1      # dtype
    assert libda.da_create(None, 4, 0, ctypes.byref(h)) == 1
    Q[0, 1] = 200                                                                             # not int8
    assert libda.da_create(Q.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(h)) == 1
    assert b"outside [-128, 127]" in libda.da_last_error()
    Qf = np.zeros((3, 3), np.float32)
    Qf[0, 2] = np.inf
    assert libda.da_create(Qf.ctypes.data_as(ctypes.c_void_p), 3, 1, ctypes.byref(h)) == 1
    assert libda.da_anneal(None, None, 0, ctypes.c_float(0), 1, 0, 0, None) == 1
    assert libda.da_words(64) == 2 and libda.da_words(65) == 3 and libda.da_words(0) == 0


def test_no_cpu_fallback(libda):
    """Without a CUDA device a valid request fails with DA_ECUDA instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p()
    Q = np.triu(np.ones((8, 8), np.int32))
    assert libda.da_create(Q.ctypes.data_as(ctypes.c_void_p), 8, 0, ctypes.byref(h)) == 6


def test_server_needs_a_device(libda):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p()
    assert libda.da_server_create(ctypes.c_int64(1 << 30), 16, ctypes.byref(h)) == 6
    assert libda.da_server_create(ctypes.c_int64(0), 16, ctypes.byref(h)) == 1


def test_failure_injection_arguments(libda):
    """The failure-injection switch validates its arguments and can be disarmed
    without a device; nothing is live before any allocation."""
    assert libda.da_diag_fail_alloc(-1, 1) == 1
    assert libda.da_diag_fail_alloc(0, -1) == 1
    assert libda.da_diag_fail_alloc(0, 0) == 0
    c, b, inj = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert libda.da_diag_live_allocations(ctypes.byref(c), ctypes.byref(b), ctypes.byref(inj)) == 0
    assert c.value >= 0 and b.value >= 0 and inj.value >= 0


def test_cancel_rejects_null(libda):
    from paper_1806_08815_gb300 import binding as b
    assert libda.da_cancel(None) == 1


def test_segment_rejects_bad_ranges_without_a_device(libda):
    """da_anneal_segment validates its arguments before touching a device."""
    assert libda.da_anneal_segment(None, None, 0, 0, 0, ctypes.c_float(0), 1, 0, 0, None, None, None) == 1


def test_batch_force_arguments(libda):
    """The batched launch's configuration override is host-only: every documented value is
    accepted (staging -1 tuner, 0 L2, 1 shared memory, 2 L2 in the warp row order), the rest
    is refused, and (-1, 0) restores the tuner."""
    libda.da_batch_force.argtypes = [ctypes.c_int32, ctypes.c_int32]
    try:
        for staging, wpb in ((-1, 0), (0, 1), (0, 4), (1, 16), (2, 0), (2, 2), (2, 4)):
            assert libda.da_batch_force(staging, wpb) == 0, (staging, wpb)
        for staging, wpb in ((3, 0), (-2, 0), (2, 8), (0, 16), (1, 1), (0, 3)):
            assert libda.da_batch_force(staging, wpb) == 1, (staging, wpb)
    finally:
        assert libda.da_batch_force(-1, 0) == 0
