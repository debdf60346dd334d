"""The fused z pass of the literal form (z forward -> exponential update with the invariant
sums -> z inverse in one kernel) at every line length the library dispatches to it, against
the FP64 oracle's literal stepping (Alg. 1 + Alg. 2 with t_end = h, repeated).

FP64 has a fused plan for powers of two (2 .. 512), FP32 also for 3 * 2^a (6 .. 384); the
z length is the only long axis, so the oracle stays cheap.  The x extent (20 in FP32, 10 in
FP64: 10 or 5 complex columns, rows of 80 bytes, a multiple of 16, so the tensor-copy variant
applies) leaves a ragged last tile for every tile width, and white noise (not divergence
free, every wavenumber populated, Nyquist planes included) exercises every coefficient.
Each test checks, through the context's kernel profile, that the fused kernel ran, then
compares each of the six fields (FP64 within 1e-12, FP32 within 1e-5 relative L2) and the
invariants of the first and last records with the oracle's physical-space values.
"""
import numpy as np
import pytest

import synth
from oracle import invariants as oinv
from oracle import scheme
from tests.gpu_util import field_rel_l2, inv_diff, inv_scales, solver_mod

pytestmark = pytest.mark.gpu

POW2 = [2, 4, 8, 16, 32, 64, 128, 256, 512]
THREE_POW2 = [6, 12, 24, 48, 96, 192, 384]
CASES = [("fp64", n) for n in POW2] + [("fp32", n) for n in POW2 + THREE_POW2]


def _run(mx, g, E0, H0, eps, mu, P, h, steps):
    import torch

    dt = torch.float64 if P == mx.MX_FP64 else torch.float32
    s = mx.Solver(g.n, g.lo, g.hi, eps, mu, P, mx.MX_FORM_LITERAL)
    try:
        Ed = torch.tensor(E0, dtype=dt, device="cuda")
        Hd = torch.tensor(H0, dtype=dt, device="cuda")
        s.load(Ed, Hd)
        s.profile(True)
        s.step(h, steps, 1)
        prof = s.profile_read()
        s.profile(False)
        s.read(Ed, Hd)
        s.sync()
        inv = s.invariants()
    finally:
        s.close()
    return Ed.double().cpu().numpy(), Hd.double().cpu().numpy(), inv, prof


@pytest.mark.parametrize("prec,nz", CASES, ids=[f"{p}-z{n}" for p, n in CASES])
def test_fused_z_length_matches_oracle(prec, nz):
    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    ny = 6 if nz >= 256 else 8
    g = synth.Grid((10 if prec == "fp64" else 20, ny, nz), (0.0, 0.0, 0.0), (2.0, 3.0, 2.5))
    rng = np.random.default_rng(1000 + nz)
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    eps, mu, h, steps = 1.6, 0.7, 0.031, 4
    E, H, inv, prof = _run(mx, g, E0, H0, eps, mu, P, h, steps)
    assert prof["z_fused"][1] == steps, f"fused z pass not used: {prof}"
    Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    tol = 1e-12 if prec == "fp64" else 1e-5
    errs = field_rel_l2(E, H, Eo, Ho)
    assert max(errs) < tol, errs
    assert len(inv) == steps + 1
    r0 = oinv.invariants(E0, H0, g.lo, g.hi, eps, mu)
    rn = oinv.invariants(Eo, Ho, g.lo, g.hi, eps, mu)
    sc = inv_scales(r0, eps, mu)
    assert inv_diff(inv[0], r0, sc) < tol
    assert inv_diff(inv[-1], rn, sc) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_z_512_commensurate_table(prec):
    """z = 512 on a cube (commensurate domain: coefficients from the per-|k|^2 table, the
    instantiation the benchmark runs) with a 64 x 64 cross-section: several tiles per row."""
    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    g = synth.Grid((64, 16, 512), (0.0, 0.0, 0.0), (2 * np.pi, 2 * np.pi, 2 * np.pi))
    rng = np.random.default_rng(77)
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    eps, mu, h, steps = 1.0, 1.0, 0.02, 3
    E, H, inv, prof = _run(mx, g, E0, H0, eps, mu, P, h, steps)
    assert prof["z_fused"][1] == steps
    Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    errs = field_rel_l2(E, H, Eo, Ho)
    assert max(errs) < (1e-12 if prec == "fp64" else 1e-5), errs
