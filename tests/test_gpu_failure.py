"""Failure detection without a GPU fault.

* A device wait that gives up: the context's fused z pass is told to give up its tile waits at
  once (mx_debug_wait_limit(ctx, 0)); each block leaves the pass after the copy it issued has
  landed, the host latches MX_E_TIMEOUT, mx_sync and every later call on the context report it,
  and the GPU stays usable (a fresh context then matches the oracle).
* Allocations that fail: mx_debug_fail_alloc(k) makes the k-th allocation of the library fail
  once.  For every k up to the number of allocations a call makes, mx_create, mx_batch_create and
  a server admission report MX_E_NOMEM and release what they had allocated (device memory back
  to where it was); the next call succeeds.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import scheme
from tests.gpu_util import max_field_rel_l2, run_gpu, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _free_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wait_limit_latches_timeout_and_gpu_stays_usable(prec):
    mx = solver_mod()
    P = mx.MX_FP32 if prec == "fp32" else mx.MX_FP64
    s = mx.Solver((64, 32, 64), (0, 0, 0), (TWO_PI,) * 3, 1.0, 1.0, P, mx.MX_FORM_LITERAL)
    s.load_random(1, 4.0)
    s.sync()
    assert mx.mx_debug_wait_limit(s.handle, 0) == mx.MX_OK
    s.profile(True)
    assert mx.mx_step(s.handle, 0.01, 2, 1) == mx.MX_OK  # enqueued; the outcome shows at the sync
    assert mx.mx_sync(s.handle) == mx.MX_E_TIMEOUT
    assert mx.mx_step(s.handle, 0.01, 1, 1) == mx.MX_E_TIMEOUT  # latched
    assert mx.mx_sync(s.handle) == mx.MX_E_TIMEOUT
    s.close()
    # the device is fine: a fresh context (default bound) runs the same pass and matches the oracle
    g = synth.Grid((16, 12, 16), (0, 0, 0), (TWO_PI,) * 3)
    rng = np.random.default_rng(3)
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    E, H, _ = run_gpu(g, E0, H0, 1.3, 0.8, P, mx.MX_FORM_LITERAL, 0.05, 3)
    Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, 1.3, 0.8, 0.05, 3)
    assert max_field_rel_l2(E, H, Eo, Ho) < (1e-12 if prec == "fp64" else 1e-5)


def test_wait_limit_default_restored():
    mx = solver_mod()
    g = synth.Grid((16, 12, 16), (0, 0, 0), (TWO_PI,) * 3)
    s = mx.Solver(g.n, g.lo, g.hi, 1.0, 1.0, mx.MX_FP32, mx.MX_FORM_LITERAL)
    s.load_random(2, 3.0)
    assert mx.mx_debug_wait_limit(s.handle, 0) == mx.MX_OK
    assert mx.mx_debug_wait_limit(s.handle, -1) == mx.MX_OK  # back to the default bound
    s.step(0.02, 3, 1)
    s.sync()
    assert len(s.invariants()) == 4
    s.close()
    assert mx.mx_debug_wait_limit(None, 0) == mx.MX_E_INVAL


def _count_failures(mx, make):
    """Arm the k-th allocation to fail for k = 0, 1, ... until `make` succeeds; every failing call
    must report MX_E_NOMEM and leave device memory as it was.  Returns the number of allocations."""
    base = _free_bytes()
    k = 0
    while True:
        assert mx.mx_debug_fail_alloc(k) == mx.MX_OK
        st, obj, close = make()
        if st == mx.MX_OK:
            mx.mx_debug_fail_alloc(-1)
            close(obj)
            return k
        assert st == mx.MX_E_NOMEM, (k, st)
        assert obj is None
        # everything allocated before the failing call was released (allocation granularity: 2 MiB)
        assert abs(_free_bytes() - base) <= 4 << 20, (k, base - _free_bytes())
        k += 1
        assert k < 64, "the armed failure never fired"


@pytest.mark.parametrize("form", ["literal", "spectral"])
def test_create_releases_everything_on_allocation_failure(form):
    mx = solver_mod()
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_SPECTRAL
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(TWO_PI, TWO_PI, TWO_PI)

    def make():
        h = C.c_void_p()
        st = mx.mx_create(C.byref(h), 128, 128, 96, lo, hi, 1.0, 1.0, mx.MX_FP32, F, None)
        return st, (h if h.value else None), mx.mx_destroy

    try:
        n = _count_failures(mx, make)
    finally:
        mx.mx_debug_fail_alloc(-1)
    # fields, spectra, table, partial sums, counter, three twiddle tables, records
    assert n >= 9
    s = mx.Solver((128, 128, 96), (0, 0, 0), (TWO_PI,) * 3, 1.0, 1.0, mx.MX_FP32, F)
    s.load_random(4, 8.0)
    s.step(0.02, 2, 1)
    s.sync()
    s.close()


def test_batch_create_releases_everything_on_allocation_failure():
    mx = solver_mod()
    specs = [dict(n=(32, 32, 32), eps=1.5, mu=2.5, h=0.031), dict(n=(48, 64, 80), eps=3.2, mu=1.1, h=0.017),
             dict(n=(64, 64, 64), eps=1.0, mu=4.0, h=0.09)]

    def make():
        try:
            b = mx.Batch(specs, mx.MX_FP32)
        except mx.MaxexpError as e:
            return e.status, None, None
        return mx.MX_OK, b, lambda b: b.close()

    try:
        n = _count_failures(mx, make)
    finally:
        mx.mx_debug_fail_alloc(-1)
    assert n >= 3 * 9 + 4
    b = mx.Batch(specs, mx.MX_FP32)
    b.load_random(7, 3.0)
    b.step(3, 1)
    b.sync()
    b.close()


def test_server_admission_reports_allocation_failure_and_keeps_serving():
    import torch

    mx = solver_mod()
    srv = mx.Server(8 << 30, max_active=4)
    try:
        n = (32, 32, 32)
        E0 = torch.randn((3,) + n, dtype=torch.float32).pin_memory()
        H0 = torch.randn((3,) + n, dtype=torch.float32).pin_memory()
        Eo, Ho = torch.empty_like(E0).pin_memory(), torch.empty_like(H0).pin_memory()
        # the worker's next allocation (the new context's first buffer) fails
        assert mx.mx_debug_fail_alloc(0) == mx.MX_OK
        rid = srv.submit(n, E0, H0, Eo, Ho, 1.0)
        assert srv.wait(rid, 60.0) == -mx.MX_E_NOMEM
        with pytest.raises(mx.MaxexpError):
            srv.result(rid)
        mx.mx_debug_fail_alloc(-1)
        rid = srv.submit(n, E0, H0, Eo, Ho, 1.0)
        assert srv.wait(rid, 60.0) == 2
        srv.result(rid)
        st = srv.stats()
        assert st["rejected"] >= 1 and st["completed"] >= 1
    finally:
        mx.mx_debug_fail_alloc(-1)
        srv.close()
