"""ctypes binding of libmaxexp (include/maxexp.h): argument marshalling only.

Every function of the C ABI is exposed under its own name (``mx_create``,
``mx_load_fields``, ``mx_step``, ...).  ``Solver`` wraps them for torch
tensors and numpy arrays; it raises on any non-OK status.  There is no CPU
fallback: importing this module fails loudly when the shared library is
missing or does not load.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MAXEXP_LIB") or os.path.join(_PKG, "lib", "libmaxexp.so")

MX_OK, MX_E_INVAL, MX_E_UNSUPPORTED_N, MX_E_NOMEM, MX_E_CUDA, MX_E_TIMEOUT, MX_E_STATE = range(7)
MX_FP64, MX_FP32 = 0, 1
MX_FORM_LITERAL, MX_FORM_SPECTRAL, MX_FORM_XY = 0, 1, 2
KERNEL_KINDS = ("x_r2c", "x_c2r", "y_fft", "z_fft", "spectral", "table", "gen", "z_fused")


class mx_instance_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("eps", C.c_double), ("mu", C.c_double), ("h", C.c_double)]


class mx_request(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("eps", C.c_double), ("mu", C.c_double), ("precision", C.c_int),
                ("t_end", C.c_double), ("nsteps", C.c_longlong), ("invariants_every", C.c_int),
                ("E0", C.c_void_p), ("H0", C.c_void_p), ("E_out", C.c_void_p), ("H_out", C.c_void_p)]


class mx_server_info(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("admitted", C.c_longlong), ("completed", C.c_longlong),
                ("rejected", C.c_longlong), ("queued", C.c_longlong), ("active", C.c_longlong),
                ("pooled_contexts", C.c_longlong), ("hbm_in_use", C.c_size_t), ("hbm_high_water", C.c_size_t),
                ("hbm_budget", C.c_size_t), ("max_concurrent", C.c_longlong), ("mean_concurrent", C.c_double),
                ("busy_s", C.c_double), ("request_s_sum", C.c_double)]


class mx_invariants(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("step", C.c_longlong),
        ("E1", C.c_double), ("E2", C.c_double),
        ("E3", C.c_double * 3), ("E4", C.c_double * 3), ("E5", C.c_double * 3), ("E6", C.c_double * 3),
        ("H1", C.c_double), ("H2", C.c_double),
        ("M1", C.c_double * 3), ("M2", C.c_double * 3),
        ("divE", C.c_double), ("divH", C.c_double),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = np.array(list(v)) if isinstance(v, C.Array) else v
        return d


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmaxexp.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python paper_2210_06232_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    P, I, D, LL, V = C.c_void_p, C.c_int, C.c_double, C.c_longlong, C.c_void_p
    D3 = C.POINTER(C.c_double)
    sig = {
        "mx_create": (I, [C.POINTER(P), I, I, I, D3, D3, D, D, I, I, V]),
        "mx_footprint_bytes": (I, [I, I, I, I, I, C.POINTER(C.c_size_t)]),
        "mx_load_fields": (I, [P, V, V, I]),
        "mx_step": (I, [P, D, LL, I]),
        "mx_read_fields": (I, [P, V, V, I]),
        "mx_read_invariants": (I, [P, C.POINTER(mx_invariants), LL, C.POINTER(LL)]),
        "mx_time": (I, [P, C.POINTER(D), C.POINTER(LL)]),
        "mx_load_random_divfree": (I, [P, C.c_ulonglong, D]),
        "mx_profile": (I, [P, I]),
        "mx_autotune": (I, [P]),
        "mx_load_fields_async": (I, [P, V, V]),
        "mx_read_fields_async": (I, [P, V, V]),
        "mx_server_create": (I, [C.POINTER(P), C.c_size_t, I]),
        "mx_server_submit": (I, [P, C.POINTER(mx_request), C.POINTER(LL)]),
        "mx_server_poll": (I, [P, LL, C.POINTER(I)]),
        "mx_server_wait": (I, [P, LL, D, C.POINTER(I)]),
        "mx_server_result": (I, [P, LL, C.POINTER(mx_invariants), LL, C.POINTER(LL), C.POINTER(D), I]),
        "mx_server_stats": (I, [P, C.POINTER(mx_server_info)]),
        "mx_server_destroy": (None, [P]),
        "mx_batch_create": (I, [C.POINTER(P), C.POINTER(mx_instance_desc), I, I, V]),
        "mx_batch_create_form": (I, [C.POINTER(P), C.POINTER(mx_instance_desc), I, I, I, V]),
        "mx_batch_size": (I, [P, C.POINTER(I)]),
        "mx_batch_instance": (I, [P, I, C.POINTER(P)]),
        "mx_batch_load_random": (I, [P, C.c_ulonglong, D]),
        "mx_batch_step": (I, [P, LL, I]),
        "mx_batch_sync": (I, [P]),
        "mx_batch_graph_used": (I, [P, C.POINTER(I)]),
        "mx_batch_launch_shape": (I, [P, C.POINTER(I), C.POINTER(I)]),
        "mx_batch_destroy": (None, [P]),
        "mx_schedule": (I, [P, C.POINTER(I), I]),
        "mx_set_schedule": (I, [P, C.POINTER(I), I]),
        "mx_spectral_update_noalloc": (I, [V, V, I, I, I, D3, D3, D, D, I, D, C.POINTER(mx_invariants), V]),
        "mx_profile_read": (I, [P, C.POINTER(D), C.POINTER(LL)]),
        "mx_debug_fail_alloc": (I, [LL]),
        "mx_debug_wait_limit": (I, [P, LL]),
        "mx_fma_peak": (I, [I, C.POINTER(D)]),
        "mx_tile_stream": (I, [V, I, I, I, I, I, C.POINTER(D)]),
        "mx_dft8_stage_eval": (I, [I, V, V, LL, I, C.POINTER(D)]),
        "mx_sync": (I, [P]),
        "mx_strerror": (C.c_char_p, [I]),
        "mx_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib, sig


_lib, _SIG = _load()
EXPORTS = tuple(_SIG)

mx_create = _lib.mx_create
mx_footprint_bytes = _lib.mx_footprint_bytes
mx_load_fields = _lib.mx_load_fields
mx_step = _lib.mx_step
mx_read_fields = _lib.mx_read_fields
mx_read_invariants = _lib.mx_read_invariants
mx_time = _lib.mx_time
mx_load_random_divfree = _lib.mx_load_random_divfree
mx_profile = _lib.mx_profile
mx_autotune = _lib.mx_autotune
mx_load_fields_async = _lib.mx_load_fields_async
mx_read_fields_async = _lib.mx_read_fields_async
mx_server_create = _lib.mx_server_create
mx_server_submit = _lib.mx_server_submit
mx_server_poll = _lib.mx_server_poll
mx_server_wait = _lib.mx_server_wait
mx_server_result = _lib.mx_server_result
mx_server_stats = _lib.mx_server_stats
mx_server_destroy = _lib.mx_server_destroy
mx_batch_create = _lib.mx_batch_create
mx_batch_create_form = _lib.mx_batch_create_form
mx_batch_size = _lib.mx_batch_size
mx_batch_instance = _lib.mx_batch_instance
mx_batch_load_random = _lib.mx_batch_load_random
mx_batch_step = _lib.mx_batch_step
mx_batch_sync = _lib.mx_batch_sync
mx_batch_graph_used = _lib.mx_batch_graph_used
mx_batch_launch_shape = _lib.mx_batch_launch_shape
mx_batch_destroy = _lib.mx_batch_destroy
mx_schedule = _lib.mx_schedule
mx_set_schedule = _lib.mx_set_schedule
mx_spectral_update_noalloc = _lib.mx_spectral_update_noalloc
mx_profile_read = _lib.mx_profile_read
mx_debug_fail_alloc = _lib.mx_debug_fail_alloc
mx_debug_wait_limit = _lib.mx_debug_wait_limit
mx_fma_peak = _lib.mx_fma_peak
mx_tile_stream = _lib.mx_tile_stream
mx_dft8_stage_eval = _lib.mx_dft8_stage_eval


def fma_peak(precision):
    """Measured FMA throughput (flop/s, an FMA counting two) of the FP64 or FP32 pipe."""
    v = C.c_double(0)
    check(mx_fma_peak(int(precision), C.byref(v)), "mx_fma_peak")
    return v.value


def tile_stream(buf_ptr, mx_, ny, nz, cols, reps=5):
    """GB/s that HBM delivers for z-line tiles of `cols` columns (rows of 8 cols bytes) of a
    [6][nz][ny][mx_] complex FP32 spectrum at device address buf_ptr (left unchanged)."""
    v = C.c_double(0)
    check(mx_tile_stream(C.c_void_p(int(buf_ptr)), int(mx_), int(ny), int(nz), int(cols), int(reps), C.byref(v)),
          "mx_tile_stream")
    return v.value
mx_sync = _lib.mx_sync
mx_strerror = _lib.mx_strerror
mx_destroy = _lib.mx_destroy


class MaxexpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {mx_strerror(status).decode()} (status {status})")


def check(status, where=""):
    if status != MX_OK:
        raise MaxexpError(status, where)


def _ptr(a, itemsize=None, count=None):
    """(address, on_device) of a torch tensor or numpy array (contiguous, checked size)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        isz, n, addr, dev = a.element_size(), a.numel(), a.data_ptr(), 1 if a.is_cuda else 0
    else:
        if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be a C-contiguous numpy array")
        isz, n, addr, dev = a.itemsize, a.size, a.ctypes.data, 0
    if itemsize is not None and isz != itemsize:
        raise ValueError(f"element size {isz} does not match the solver precision ({itemsize} bytes)")
    if count is not None and n != count:
        raise ValueError(f"array has {n} elements, expected {count}")
    return addr, dev


def footprint_bytes(n, precision=MX_FP64, form=MX_FORM_LITERAL):
    out = C.c_size_t(0)
    check(mx_footprint_bytes(int(n[0]), int(n[1]), int(n[2]), int(precision), int(form), C.byref(out)),
          "mx_footprint_bytes")
    return int(out.value)


class Solver:
    """One grid, one (eps, mu), one precision and form: a libmaxexp context."""

    def __init__(self, n, lo, hi, eps, mu, precision=MX_FP64, form=MX_FORM_LITERAL, stream=None):
        self.n = tuple(int(v) for v in n)
        self.precision = precision
        self.form = form
        self.dtype = np.float64 if precision == MX_FP64 else np.float32
        lo3 = (C.c_double * 3)(*lo)
        hi3 = (C.c_double * 3)(*hi)
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        check(mx_create(C.byref(h), *self.n, lo3, hi3, float(eps), float(mu), int(precision), int(form), s),
              "mx_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            mx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _fields(self, E, H):
        isz = 8 if self.precision == MX_FP64 else 4
        cnt = 3 * self.n[0] * self.n[1] * self.n[2]
        pe, de = _ptr(E, isz, cnt)
        ph, dh = _ptr(H, isz, cnt)
        return pe, de, ph, dh

    def load(self, E, H):
        pe, de, ph, dh = self._fields(E, H)
        if de != dh:
            raise ValueError("E and H must both be on the host or both on the device")
        self._keep = (E, H)
        check(mx_load_fields(self._h, pe, ph, de), "mx_load_fields")

    def step(self, h, nsteps=1, invariants_every=1):
        check(mx_step(self._h, float(h), int(nsteps), int(invariants_every)), "mx_step")

    def read(self, E, H):
        pe, de, ph, dh = self._fields(E, H)
        if de != dh:
            raise ValueError("E and H must both be on the host or both on the device")
        check(mx_read_fields(self._h, pe, ph, de), "mx_read_fields")
        return E, H

    def read_numpy(self):
        shape = (3, self.n[2], self.n[1], self.n[0])
        E = np.empty(shape, self.dtype)
        H = np.empty(shape, self.dtype)
        return self.read(E, H)

    def invariants(self, max_records=None):
        if max_records is None:
            cnt = C.c_longlong(0)
            check(mx_read_invariants(self._h, None, 0, C.byref(cnt)), "mx_read_invariants")
            max_records = cnt.value
        if max_records == 0:
            return []
        buf = (mx_invariants * int(max_records))()
        n = C.c_longlong(0)
        check(mx_read_invariants(self._h, buf, int(max_records), C.byref(n)), "mx_read_invariants")
        return [buf[i].as_dict() for i in range(n.value)]

    def load_random(self, seed, sigma):
        check(mx_load_random_divfree(self._h, int(seed), float(sigma)), "mx_load_random_divfree")

    def autotune(self):
        check(mx_autotune(self._h), "mx_autotune")

    SCHEDULE_PASSES = ("x_r2c", "y_fwd", "z_fwd", "z_inv", "y_inv", "x_c2r", "z_fused")
    SCHEDULE_VARIANTS = ("copy-engine", "register-prefetch", "copy-engine-2stage")

    def schedule(self):
        """{pass: (blocks per SM, 'copy-engine' | 'register-prefetch' | 'copy-engine-2stage')} in use."""
        arr = (C.c_int * 7)()
        check(mx_schedule(self._h, arr, 7), "mx_schedule")
        return {p: (v & 15, self.SCHEDULE_VARIANTS[min(v >> 4, 2)]) for p, v in zip(self.SCHEDULE_PASSES, arr)}

    def set_schedule(self, sched):
        """Set the schedules of this shape: {pass: (blocks per SM, variant name)}, every pass given."""
        arr = (C.c_int * 7)()
        for i, p in enumerate(self.SCHEDULE_PASSES):
            bps, name = sched[p]
            arr[i] = int(bps) + 16 * self.SCHEDULE_VARIANTS.index(name)
        check(mx_set_schedule(self._h, arr, 7), "mx_set_schedule")

    def profile(self, enable=True):
        check(mx_profile(self._h, 1 if enable else 0), "mx_profile")

    def profile_read(self):
        n = len(KERNEL_KINDS)
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        check(mx_profile_read(self._h, ms, cnt), "mx_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}

    def time(self):
        t = C.c_double(0)
        s = C.c_longlong(0)
        check(mx_time(self._h, C.byref(t), C.byref(s)), "mx_time")
        return t.value, s.value

    def sync(self):
        check(mx_sync(self._h), "mx_sync")


class _Borrowed(Solver):
    """A context owned by a batch: same methods as Solver, never destroyed here."""

    def __init__(self, handle, n, precision, form=MX_FORM_SPECTRAL):
        self._h = handle
        self.n = n
        self.precision = precision
        self.form = form
        self.dtype = np.float64 if precision == MX_FP64 else np.float32

    def close(self):
        self._h = C.c_void_p()


class Batch:
    """Independent spectral-form instances advanced by one persistent launch per step call."""

    def __init__(self, instances, precision=MX_FP32, stream=None, form=MX_FORM_SPECTRAL):
        """instances: list of dicts with keys n=(nx,ny,nz), lo, hi, eps, mu, h; form MX_FORM_SPECTRAL
        (one persistent launch per step call), MX_FORM_LITERAL or MX_FORM_XY (graph of per-instance pass
        chains)."""
        arr = (mx_instance_desc * len(instances))()
        for i, d in enumerate(instances):
            arr[i].nx, arr[i].ny, arr[i].nz = (int(v) for v in d["n"])
            arr[i].lo = (C.c_double * 3)(*d.get("lo", (0.0, 0.0, 0.0)))
            arr[i].hi = (C.c_double * 3)(*d.get("hi", (2 * np.pi,) * 3))
            arr[i].eps, arr[i].mu, arr[i].h = float(d["eps"]), float(d["mu"]), float(d["h"])
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        check(mx_batch_create_form(C.byref(h), arr, len(instances), int(precision), int(form), s), "mx_batch_create")
        self._h = h
        self.precision = precision
        self.form = form
        self.specs = [dict(d) for d in instances]

    def __len__(self):
        return len(self.specs)

    def instance(self, i):
        c = C.c_void_p()
        check(mx_batch_instance(self._h, int(i), C.byref(c)), "mx_batch_instance")
        return _Borrowed(c, tuple(int(v) for v in self.specs[i]["n"]), self.precision, self.form)

    def load_random(self, seed, sigma):
        check(mx_batch_load_random(self._h, int(seed), float(sigma)), "mx_batch_load_random")

    def step(self, nsteps, invariants_every=1):
        check(mx_batch_step(self._h, int(nsteps), int(invariants_every)), "mx_batch_step")

    def sync(self):
        check(mx_batch_sync(self._h), "mx_batch_sync")

    def graph_used(self):
        """1: replayed from a captured graph; 0: not yet; -e: capture refused with CUDA error e."""
        v = C.c_int(0)
        check(mx_batch_graph_used(self._h, C.byref(v)), "mx_batch_graph_used")
        return v.value

    def launch_shape(self):
        """(blocks, threads per block) of the spectral form's persistent launch; (0, 0) for the literal form."""
        nb, nt = C.c_int(0), C.c_int(0)
        check(mx_batch_launch_shape(self._h, C.byref(nb), C.byref(nt)), "mx_batch_launch_shape")
        return nb.value, nt.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            mx_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (native worker thread in libmaxexp)."""

    def __init__(self, hbm_budget_bytes, max_active=64):
        h = C.c_void_p()
        check(mx_server_create(C.byref(h), int(hbm_budget_bytes), int(max_active)), "mx_server_create")
        self._h = h
        self._keep = {}

    def submit(self, n, E0, H0, E_out, H_out, t_end, eps=1.0, mu=1.0, precision=MX_FP32, nsteps=1,
               invariants_every=0, lo=(0.0, 0.0, 0.0), hi=(2 * np.pi,) * 3):
        """Host buffers (pinned torch tensors or numpy arrays) stay borrowed until the request is done."""
        isz = 8 if precision == MX_FP64 else 4
        cnt = 3 * int(n[0]) * int(n[1]) * int(n[2])
        bufs = [_ptr(a, isz, cnt) for a in (E0, H0, E_out, H_out)]
        if any(d for _, d in bufs):
            raise ValueError("server requests take host buffers")
        r = mx_request()
        r.nx, r.ny, r.nz = (int(v) for v in n)
        r.lo = (C.c_double * 3)(*lo)
        r.hi = (C.c_double * 3)(*hi)
        r.eps, r.mu, r.precision = float(eps), float(mu), int(precision)
        r.t_end, r.nsteps, r.invariants_every = float(t_end), int(nsteps), int(invariants_every)
        r.E0, r.H0, r.E_out, r.H_out = (b for b, _ in bufs)
        rid = C.c_longlong(0)
        check(mx_server_submit(self._h, C.byref(r), C.byref(rid)), "mx_server_submit")
        self._keep[rid.value] = (E0, H0, E_out, H_out)
        return rid.value

    def poll(self, rid):
        st = C.c_int(0)
        check(mx_server_poll(self._h, int(rid), C.byref(st)), "mx_server_poll")
        return st.value

    def wait(self, rid, timeout=60.0):
        st = C.c_int(0)
        s = mx_server_wait(self._h, int(rid), float(timeout), C.byref(st))
        if s not in (MX_OK, MX_E_TIMEOUT):
            check(s, "mx_server_wait")
        return st.value

    def result(self, rid, release=True):
        """(invariant records, latency in seconds) of a done request."""
        n = C.c_longlong(0)
        lat = C.c_double(0)
        check(mx_server_result(self._h, int(rid), None, 0, C.byref(n), None, 0), "mx_server_result")
        buf = (mx_invariants * max(1, n.value))()
        check(mx_server_result(self._h, int(rid), buf, n.value, C.byref(n), C.byref(lat), 1 if release else 0),
              "mx_server_result")
        if release:
            self._keep.pop(int(rid), None)
        return [buf[i].as_dict() for i in range(n.value)], lat.value

    def stats(self):
        info = mx_server_info()
        check(mx_server_stats(self._h, C.byref(info)), "mx_server_stats")
        return {name: getattr(info, name) for name, _ in info._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            mx_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
