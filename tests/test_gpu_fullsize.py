"""Parity at the benchmark's full sizes.

* 128 x 256 x 128 on [0,2pi] x [0,4pi] x [0,2pi], FP64, eps = 2, mu = 1, random
  divergence-free fields (sigma = 8), h = 0.05, 1000 steps, invariants every step:
  element by element against the oracle (one step of size 1000 h, equal to the repeated step
  to round-off by the group property).
* 512^3 (the bench grid, the bench's kernels and launch shapes): a sum of plane waves, 500
  steps of h = 0.02; sampled outputs against the closed form: the literal FP32 form (the
  benchmarked step), the spectral-resident form in FP32 and FP64.
"""
import numpy as np
import pytest

import synth
from oracle import closed_form as cf
from oracle import scheme
from tests.gpu_util import inv_diff, inv_scales, rel_l2, solver_mod

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["spectral", "literal"])
def test_random_128x256x128_1000_steps_fp64(form):
    import torch

    mx = solver_mod()
    g = synth.Grid((128, 256, 128), (0, 0, 0), (2 * np.pi, 4 * np.pi, 2 * np.pi))
    E0, H0 = synth.random_divfree_fields(g, seed=2, sigma=8.0)
    eps, mu, h, n = 2.0, 1.0, 0.05, 1000
    F = mx.MX_FORM_SPECTRAL if form == "spectral" else mx.MX_FORM_LITERAL
    s = mx.Solver(g.n, g.lo, g.hi, eps, mu, mx.MX_FP64, F)
    Ed, Hd = torch.tensor(E0, device="cuda"), torch.tensor(H0, device="cuda")
    s.load(Ed, Hd)
    s.step(h, n, 1)
    s.read(Ed, Hd)
    s.sync()
    inv = s.invariants()
    s.close()
    Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, n * h)
    assert rel_l2(Ed.cpu().numpy(), Hd.cpu().numpy(), Eo, Ho) < 1e-12
    assert len(inv) == n + 1
    sc = inv_scales(inv[0], eps, mu)
    # 1e-13 relative drift in both forms.  The spectral form evaluates R(t_n) directly (nothing
    # accumulates); the literal form re-applies the same transforms and R(h) every step, and keeps
    # within the bound because its FFT rotations are lifted (determinant 1 whatever the rounding of
    # their constants) and its other constants double-double pairs (with FP64-rounded constants it
    # drifted 3.2e-13 over these 1000 steps).
    drift = max(inv_diff(r, inv[0], sc) for r in inv)
    print(form, "max normalised invariant drift over", n, "steps:", drift)
    assert drift < 1e-13


def _plane_wave_device(torch, n, params, dtype):
    """E0, H0 of a plane-wave sum evaluated on the device (input construction only)."""
    ax = torch.arange(n, device="cuda", dtype=torch.float64) * (2 * np.pi / n)
    z, y, x = torch.meshgrid(ax, ax, ax, indexing="ij")
    E = torch.zeros((3, n, n, n), device="cuda", dtype=torch.float64)
    H = torch.zeros_like(E)
    for kj, aj, pj, wj in zip(params["k"], params["a"], params["phi"], params["omega"]):
        ph = torch.cos(kj[0] * x + kj[1] * y + kj[2] * z + pj)
        bj = np.cross(kj, aj) / (params["mu"] * wj)
        for c in range(3):
            E[c] += float(aj[c]) * ph
            H[c] += float(bj[c]) * ph
        del ph
    del x, y, z
    return E.to(dtype).contiguous(), H.to(dtype).contiguous()


@pytest.mark.parametrize("prec,form", [("fp32", "literal"), ("fp32", "spectral"), ("fp64", "spectral")])
def test_512_plane_waves_sampled(prec, form):
    import torch

    mx = solver_mod()
    n, h, steps = 512, 0.02, 500
    params = synth.plane_wave_params(7, nwaves=8, kmax=40)
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    E, H = _plane_wave_device(torch, n, params, dt)
    F = mx.MX_FORM_SPECTRAL if form == "spectral" else mx.MX_FORM_LITERAL
    s = mx.Solver((n, n, n), (0, 0, 0), (2 * np.pi,) * 3, 1.0, 1.0, P, F)
    s.load(E, H)
    s.step(h, steps, 50)
    s.read(E, H)
    s.sync()
    inv = s.invariants()
    s.close()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, size=(4096, 3))  # (iz, iy, ix)
    pts = idx * (2 * np.pi / n)
    Ee, He = cf.plane_wave_sum(pts[:, 2], pts[:, 1], pts[:, 0], steps * h, params)
    sel = torch.tensor(idx, device="cuda")
    Eg = E[:, sel[:, 0], sel[:, 1], sel[:, 2]].double().cpu().numpy()
    Hg = H[:, sel[:, 0], sel[:, 1], sel[:, 2]].double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel_l2(Eg, Hg, Ee, He) < tol
    e1 = cf.plane_wave_energy(params)
    assert max(abs(r["E1"] - e1) for r in inv) < (1e-12 if prec == "fp64" else 1e-6) * e1
    del E, H
    torch.cuda.empty_cache()
