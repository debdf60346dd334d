"""The allocation-free entry point (mx_spectral_update_noalloc) against the
context path (mx_create / mx_load_fields / mx_step / mx_read_*).

Callers that cannot allocate device memory (another framework's pool,
stream recording, fixed-buffer embeddings) use mx_spectral_update_noalloc on
a spectrum they own; its scratch is a static device array shared by all
calls.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tests.gpu_util import inv_diff, inv_scales, solver_mod

pytestmark = pytest.mark.gpu


def _packed(E, H):
    """Unnormalised 3D DFT of the six fields in the packed half-spectrum layout."""
    F = np.fft.rfftn(np.concatenate([E, H]), axes=(1, 2, 3))
    m = E.shape[-1] // 2
    P = F[..., :m].copy()
    P[..., 0] = F[..., 0] + 1j * F[..., m]
    return P


def _rel(a, b):
    return np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_context_path_two_calls(prec):
    import torch

    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    g = synth.Grid((24, 20, 16), (0.0, 0.0, 0.0), (2.0, 1.7, 1.3))
    rng = np.random.default_rng(21)
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    eps, mu, h = 1.7, 0.6, 0.043

    # context path: two steps, fields after each
    s = mx.Solver(g.n, g.lo, g.hi, eps, mu, P, mx.MX_FORM_SPECTRAL)
    Ed = torch.tensor(E0, dtype=rdt, device="cuda")
    Hd = torch.tensor(H0, dtype=rdt, device="cuda")
    s.load(Ed, Hd)
    ref_fields = []
    for _ in range(2):
        s.step(h, 1, 1)
        Eo, Ho = torch.empty_like(Ed), torch.empty_like(Hd)
        s.read(Eo, Ho)
        s.sync()
        ref_fields.append((Eo.double().cpu().numpy(), Ho.double().cpu().numpy()))
    recs = s.invariants()
    s.close()
    assert len(recs) == 3

    # allocation-free path on a caller-owned spectrum, two calls in a row
    lo = (C.c_double * 3)(*g.lo)
    hi = (C.c_double * 3)(*g.hi)
    spec0 = torch.tensor(_packed(E0, H0), dtype=cdt, device="cuda")
    for i in (1, 2):
        out = torch.empty_like(spec0)
        inv = mx.mx_invariants()
        st = mx.mx_spectral_update_noalloc(spec0.data_ptr(), out.data_ptr(), *g.n, lo, hi, eps, mu, P, i * h,
                                           C.byref(inv), None)
        assert st == mx.MX_OK, mx.mx_strerror(st)
        torch.cuda.synchronize()
        got = inv.as_dict()
        sc = inv_scales(recs[0], eps, mu)
        assert inv_diff(got, recs[i], sc) < tol
        Er, Hr = ref_fields[i - 1]
        assert _rel(out.cpu().numpy().astype(np.complex128), _packed(Er, Hr)) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_modes_and_in_place(prec):
    """The other documented modes on the same grid: invariants of the input only (spec_out NULL),
    the update only (inv_out NULL), and the update in place (spec_out == spec_in)."""
    import torch

    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    tol = 1e-12 if prec == "fp64" else 1e-5
    g = synth.Grid((24, 20, 16), (0.0, 0.0, 0.0), (2.0, 1.7, 1.3))
    rng = np.random.default_rng(22)
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    eps, mu, h = 1.7, 0.6, 0.043
    lo = (C.c_double * 3)(*g.lo)
    hi = (C.c_double * 3)(*g.hi)
    spec0 = torch.tensor(_packed(E0, H0), dtype=cdt, device="cuda")

    # out of place, update and invariants: the result the other modes are compared with
    ref = torch.empty_like(spec0)
    inv_ref = mx.mx_invariants()
    assert mx.mx_spectral_update_noalloc(spec0.data_ptr(), ref.data_ptr(), *g.n, lo, hi, eps, mu, P, h,
                                         C.byref(inv_ref), None) == mx.MX_OK
    # invariants of the input only: the invariants are conserved, so they equal the updated state's
    inv0 = mx.mx_invariants()
    assert mx.mx_spectral_update_noalloc(spec0.data_ptr(), None, *g.n, lo, hi, eps, mu, P, h,
                                         C.byref(inv0), None) == mx.MX_OK
    sc = inv_scales(inv_ref.as_dict(), eps, mu)
    assert inv_diff(inv0.as_dict(), inv_ref.as_dict(), sc) < tol
    # update only
    out = torch.empty_like(spec0)
    assert mx.mx_spectral_update_noalloc(spec0.data_ptr(), out.data_ptr(), *g.n, lo, hi, eps, mu, P, h,
                                         None, None) == mx.MX_OK
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)) < tol
    # in place
    buf = spec0.clone()
    inv_ip = mx.mx_invariants()
    assert mx.mx_spectral_update_noalloc(buf.data_ptr(), buf.data_ptr(), *g.n, lo, hi, eps, mu, P, h,
                                         C.byref(inv_ip), None) == mx.MX_OK
    torch.cuda.synchronize()
    assert _rel(buf.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)) < tol
    assert inv_diff(inv_ip.as_dict(), inv_ref.as_dict(), sc) < tol


def test_noalloc_rejects_misaligned_and_capture():
    """A spectrum view that does not start on a 16-byte boundary is refused before anything is
    enqueued; so is a request for invariants while the stream is being captured."""
    import torch

    mx = solver_mod()
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    inv = mx.mx_invariants()
    spec = torch.zeros(6 * 8 * 8 * 4 + 1, dtype=torch.complex64, device="cuda")
    off = spec[1:]  # 8-byte offset
    assert mx.mx_spectral_update_noalloc(off.data_ptr(), spec.data_ptr(), 8, 8, 8, lo, hi, 1.0, 1.0, mx.MX_FP32, 0.1,
                                         C.byref(inv), None) == mx.MX_E_INVAL
    assert mx.mx_spectral_update_noalloc(spec.data_ptr(), off.data_ptr(), 8, 8, 8, lo, hi, 1.0, 1.0, mx.MX_FP32, 0.1,
                                         None, None) == mx.MX_E_INVAL
    # a capture that records nothing of ours: the call with invariants is refused before it enqueues
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = mx.mx_spectral_update_noalloc(spec.data_ptr(), spec.data_ptr(), 8, 8, 8, lo, hi, 1.0, 1.0, mx.MX_FP32,
                                           0.1, C.byref(inv), C.c_void_p(s.cuda_stream))
        spec.add_(0)  # the capture holds one node of its own
    assert st == mx.MX_E_INVAL


def test_noalloc_rejects_bad_arguments():
    mx = solver_mod()
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    inv = mx.mx_invariants()
    assert mx.mx_spectral_update_noalloc(None, None, 8, 8, 8, lo, hi, 1.0, 1.0, 0, 0.1, C.byref(inv), None) == mx.MX_E_INVAL
    dummy = C.c_void_p(1 << 20)  # 16-byte aligned, never dereferenced: validation fails first
    assert mx.mx_spectral_update_noalloc(dummy, dummy, 7, 8, 8, lo, hi, 1.0, 1.0, 0, 0.1, C.byref(inv), None) == mx.MX_E_INVAL
    assert mx.mx_spectral_update_noalloc(dummy, dummy, 8, 8, 8, lo, hi, -1.0, 1.0, 0, 0.1, C.byref(inv), None) == mx.MX_E_INVAL
    assert mx.mx_spectral_update_noalloc(dummy, dummy, 8, 8, 8, lo, hi, 1.0, 1.0, 0, float("inf"), C.byref(inv), None) == mx.MX_E_INVAL
    big = 1 << 12  # (4096/2) * 4096 * 512 = 2^32 points per component: beyond the 32-bit index range
    assert mx.mx_spectral_update_noalloc(dummy, dummy, big, big, 512, lo, hi, 1.0, 1.0, 1, 0.1, C.byref(inv), None) == \
        mx.MX_E_UNSUPPORTED_N
