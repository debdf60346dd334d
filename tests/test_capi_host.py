"""Host-side checks of libmaxexp that need no GPU: the library loads, exports
every function include/maxexp.h declares, and validates arguments before any
CUDA call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2210_06232_gb300 import maxexp

    return maxexp


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mx_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    mx = _lib()
    lib = C.CDLL(mx.LIB_PATH)
    declared = _declared()
    assert "mx_create" in declared and "mx_step" in declared
    for name in declared:
        assert hasattr(lib, name), name
        assert name in mx.EXPORTS, f"{name} has no binding"


def test_argument_validation_without_gpu():
    mx = _lib()
    h = C.c_void_p()
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    bad = [
        (7, 8, 8, 1.0, 1.0, 0, 0),      # odd
        (8, 0, 8, 1.0, 1.0, 0, 0),      # empty
        (8, 8, 8, -1.0, 1.0, 0, 0),     # eps <= 0
        (8, 8, 8, 1.0, float("nan"), 0, 0),
        (8, 8, 8, 1.0, 1.0, 5, 0),      # precision
        (8, 8, 8, 1.0, 1.0, 0, 9),      # form
    ]
    for nx, ny, nz, eps, mu, p, f in bad:
        assert mx.mx_create(C.byref(h), nx, ny, nz, lo, hi, eps, mu, p, f, None) == mx.MX_E_INVAL
        assert not h.value
    for nx, ny, nz in [(14, 8, 8), (8, 14, 8), (8, 8, 1024), (1026, 8, 8)]:
        assert mx.mx_create(C.byref(h), nx, ny, nz, lo, hi, 1.0, 1.0, 0, 0, None) == mx.MX_E_UNSUPPORTED_N
    # the xy-resident form needs a fused z plan: 10 (5 * 2) has none; 6 has one in FP32 only
    for nz, p in [(10, 1), (10, 0), (6, 0)]:
        assert mx.mx_create(C.byref(h), 8, 8, nz, lo, hi, 1.0, 1.0, p, mx.MX_FORM_XY, None) == mx.MX_E_UNSUPPORTED_N
        assert not h.value
    hi_bad = (C.c_double * 3)(1, 0, 1)
    assert mx.mx_create(C.byref(h), 8, 8, 8, lo, hi_bad, 1.0, 1.0, 0, 0, None) == mx.MX_E_INVAL
    assert mx.mx_create(None, 8, 8, 8, lo, hi, 1.0, 1.0, 0, 0, None) == mx.MX_E_INVAL
    assert mx.mx_step(None, 0.1, 1, 1) == mx.MX_E_INVAL
    mx.mx_destroy(None)
    for s in range(7):
        assert len(mx.mx_strerror(s)) > 0


def test_footprint_is_host_only_and_scales():
    mx = _lib()
    b64 = mx.footprint_bytes((512, 512, 512), mx.MX_FP64, mx.MX_FORM_SPECTRAL)
    b32 = mx.footprint_bytes((512, 512, 512), mx.MX_FP32, mx.MX_FORM_SPECTRAL)
    # the xy-resident form holds the same three field-sized buffers as the spectral one
    assert mx.footprint_bytes((512, 512, 512), mx.MX_FP32, mx.MX_FORM_XY) == b32
    assert mx.footprint_bytes((512, 512, 512), mx.MX_FP32, mx.MX_FORM_LITERAL) < b32
    assert b64 > 18 * 512 ** 3 * 8 * 0.99 and b32 < b64
    with pytest.raises(mx.MaxexpError):
        mx.footprint_bytes((7, 8, 8))


def test_schedule_calls_validate_without_gpu():
    mx = _lib()
    arr = (C.c_int * 7)(*([4] * 7))
    assert mx.mx_schedule(None, arr, 7) == mx.MX_E_INVAL
    assert mx.mx_set_schedule(None, arr, 7) == mx.MX_E_INVAL
    assert mx.mx_autotune(None) == mx.MX_E_INVAL
    assert mx.Solver.SCHEDULE_VARIANTS.index("copy-engine-2stage") == 2  # code = bps + 16 * variant


def test_noalloc_alignment_checked_before_any_cuda_call():
    """Spectrum pointers that are not 16-byte aligned are refused by the host-side checks (the
    values are never dereferenced)."""
    mx = _lib()
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    a, m = C.c_void_p(1 << 20), C.c_void_p((1 << 20) + 8)
    for p_in, p_out in ((m, a), (a, m), (m, None)):
        assert mx.mx_spectral_update_noalloc(p_in, p_out, 8, 8, 8, lo, hi, 1.0, 1.0, mx.MX_FP32, 0.1, None,
                                             None) == mx.MX_E_INVAL


def test_debug_calls_validate_without_gpu():
    """The failure-injection calls: arming and disarming the allocation fault needs no device; the
    wait limit needs a context."""
    mx = _lib()
    assert mx.mx_debug_fail_alloc(5) == mx.MX_OK
    assert mx.mx_debug_fail_alloc(-1) == mx.MX_OK
    assert mx.mx_debug_wait_limit(None, 0) == mx.MX_E_INVAL
