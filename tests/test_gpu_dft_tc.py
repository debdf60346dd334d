"""The DFT-as-GEMM evaluation (mx_dft8_stage_eval): every variant (FMA butterfly; tensor cores
with 1, 3 or 6 products of TF32-split operands) computes `reps` radix-8 stages (twiddle, then the
8-point DFT of the paper's Sec. 2.3 with the exp(-2 pi i / 8) kernel) of 128-vector tiles; the
result is compared with the same stages in FP64 (numpy, the DFT written from its definition).
The bounds follow each variant's arithmetic: FP32 for the butterfly and the 6-product split,
about 2^-21 per stage for 3 products, TF32 (2^-11) for 1."""
import numpy as np
import pytest

from tests.gpu_util import solver_mod

pytestmark = pytest.mark.gpu

BOUNDS = {0: 2e-6, 6: 2e-6, 3: 2e-5, 1: 2e-2}


def _reference(x, reps):
    """FP64 stages with the library's FP32 twiddles: w_k = fl32(exp(-2 pi i (k+1)/64) / sqrt(8))."""
    k = np.arange(8)
    a = -2.0 * np.pi * (k + 1) / 64.0
    s = 1.0 / np.sqrt(8.0)
    w = (np.cos(a) * s).astype(np.float32).astype(np.float64) + 1j * (np.sin(a) * s).astype(np.float32).astype(np.float64)
    F = np.exp(-2j * np.pi * np.outer(k, k) / 8)  # (F_8)_{kn} = exp(-2 pi i kn / 8)
    y = x.astype(np.complex128)
    for _ in range(reps):
        y = (y * w) @ F.T
    return y


@pytest.mark.parametrize("variant", [0, 1, 3, 6])
def test_dft8_stage_variants_match_fp64(variant):
    import ctypes as C

    import torch

    mx = solver_mod()
    tiles, reps = 3, 5
    rng = np.random.default_rng(8)
    x = (rng.standard_normal((tiles * 128, 8)) + 1j * rng.standard_normal((tiles * 128, 8))).astype(np.complex64)
    xin = torch.tensor(x, device="cuda")
    out = torch.empty_like(xin)
    ms = C.c_double(0)
    st = mx.mx_dft8_stage_eval(variant, xin.data_ptr(), out.data_ptr(), tiles, reps, C.byref(ms))
    assert st == mx.MX_OK, mx.mx_strerror(st)
    y = out.cpu().numpy().astype(np.complex128)
    ref = _reference(x, reps)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print(f"variant {variant}: rel L2 {err:.2e}, {ms.value:.4f} ms")
    assert err < BOUNDS[variant]
    assert ms.value > 0


def test_dft8_stage_rejects_bad_arguments():
    import ctypes as C

    mx = solver_mod()
    ms = C.c_double(0)
    p = C.c_void_p(1 << 20)
    assert mx.mx_dft8_stage_eval(2, p, p, 1, 1, C.byref(ms)) == mx.MX_E_INVAL
    assert mx.mx_dft8_stage_eval(0, p, p, 0, 1, C.byref(ms)) == mx.MX_E_INVAL
    assert mx.mx_dft8_stage_eval(0, C.c_void_p((1 << 20) + 8), p, 1, 1, C.byref(ms)) == mx.MX_E_INVAL
