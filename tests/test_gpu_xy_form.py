"""The xy-resident form (MX_FORM_XY): the literal step's map (Alg. 2 with t_end = h per step, Def.
2.3) with the state kept as the x-y spectrum, one fused z pass per step.

Against the FP64 oracle's literal stepping per field (FP64 1e-12, FP32 1e-5) and its
physical-space invariants; reads leave the state unchanged (bit for bit); the same map as the
literal form to rounding.  Grids cover nz a power of two (the 1/nz of the z pass exact), 3 * 2^a
(FP32 only; 1/nz rounded), Mx odd (no tensor copies: per-thread loads), ragged tiles.
"""
import numpy as np
import pytest

import synth
from oracle import invariants as oinv
from oracle import scheme
from tests.gpu_util import inv_diff, inv_scales, max_field_rel_l2, run_gpu, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
GRIDS = [
    ((16, 12, 32), (TWO_PI, TWO_PI, TWO_PI), ("fp64", "fp32")),
    ((10, 8, 512), (1.0, 2.0, 3.0), ("fp64", "fp32")),        # Mx = 5; direct coefficients
    ((12, 6, 384), (TWO_PI, TWO_PI, TWO_PI), ("fp32",)),       # 1/nz rounded
    ((20, 10, 48), (3.0, 1.5, 3.0), ("fp32",)),
    ((12, 16, 64), (TWO_PI, 2 * TWO_PI, TWO_PI), ("fp64", "fp32")),
]
CASES = [(gi, p) for gi, (_, _, precs) in enumerate(GRIDS) for p in precs]


def _fields(g, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)


@pytest.mark.parametrize("gi,prec", CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("device", [True, False], ids=["device", "host"])
def test_xy_form_matches_oracle(gi, prec, device):
    mx = solver_mod()
    n, hi, _ = GRIDS[gi]
    g = synth.Grid(n, (0.0, 0.0, 0.0), hi)
    E0, H0 = _fields(g, seed=40 + gi)
    eps, mu, h, steps = 1.7, 0.6, 0.043, 5
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    E, H, inv = run_gpu(g, E0, H0, eps, mu, P, mx.MX_FORM_XY, h, steps, every=1, device=device)
    Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert max_field_rel_l2(E, H, Eo, Ho) < tol
    assert len(inv) == steps + 1
    r0 = oinv.invariants(E0, H0, g.lo, g.hi, eps, mu)
    rn = oinv.invariants(Eo, Ho, g.lo, g.hi, eps, mu)
    sc = inv_scales(r0, eps, mu)
    assert inv_diff(inv[0], r0, sc) < tol
    assert inv_diff(inv[-1], rn, sc) < tol
    assert inv[-1]["step"] == steps


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_xy_form_reads_leave_the_state_unchanged(prec):
    import torch

    mx = solver_mod()
    g = synth.Grid((16, 12, 32), (0.0, 0.0, 0.0), (TWO_PI, TWO_PI, TWO_PI))
    E0, H0 = _fields(g, seed=47)
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32

    def solver():
        s = mx.Solver(g.n, g.lo, g.hi, 1.3, 0.8, P, mx.MX_FORM_XY)
        s.load(torch.tensor(E0, dtype=dt, device="cuda"), torch.tensor(H0, dtype=dt, device="cuda"))
        return s

    def read(s):
        E = torch.empty((3,) + g.shape, dtype=dt, device="cuda")
        H = torch.empty_like(E)
        s.read(E, H)
        s.sync()
        return E.cpu().numpy(), H.cpu().numpy()

    a, b = solver(), solver()
    try:
        a.step(0.05, 3, 1)
        first = read(a)
        second = read(a)
        assert np.array_equal(first[0], second[0]) and np.array_equal(first[1], second[1])
        a.step(0.05, 2, 1)
        b.step(0.05, 5, 1)
        ra, rb = read(a), read(b)
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_xy_form_is_the_literal_map(prec):
    # 64^3, 50 steps: the two forms apply the same R(h) per step; they differ only by the x and y
    # transforms the literal form runs (and rounds) every step
    mx = solver_mod()
    g = synth.Grid((64, 64, 64), (0.0, 0.0, 0.0), (TWO_PI, TWO_PI, TWO_PI))
    E0, H0 = synth.random_divfree_fields(g, seed=48, sigma=16.0)
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    lit = run_gpu(g, E0, H0, 1.0, 1.0, P, mx.MX_FORM_LITERAL, 0.02, 50, every=10)
    xy = run_gpu(g, E0, H0, 1.0, 1.0, P, mx.MX_FORM_XY, 0.02, 50, every=10)
    assert max_field_rel_l2(xy[0], xy[1], lit[0], lit[1]) < (1e-12 if prec == "fp64" else 1e-5)
    for a, b in zip(lit[2], xy[2]):
        assert abs(a["E1"] - b["E1"]) <= (1e-13 if prec == "fp64" else 1e-6) * abs(a["E1"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_xy_form_random_load_and_autotune_match_the_spectral_form(prec):
    # mx_load_random_divfree and mx_autotune in the xy-resident form: n steps of h equal the
    # spectral-resident form's R(n h) applied to the same generated spectrum (group property)
    import torch

    mx = solver_mod()
    g = synth.Grid((32, 16, 64), (0.0, 0.0, 0.0), (TWO_PI, TWO_PI, TWO_PI))
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = []
    for F in (mx.MX_FORM_XY, mx.MX_FORM_SPECTRAL):
        s = mx.Solver(g.n, g.lo, g.hi, 1.4, 0.9, P, F)
        try:
            s.autotune()
            s.load_random(11, 6.0)
            s.step(0.03, 20, 5)
            E = torch.empty((3,) + g.shape, dtype=dt, device="cuda")
            H = torch.empty_like(E)
            s.read(E, H)
            s.sync()
            out.append((E.double().cpu().numpy(), H.double().cpu().numpy(), s.invariants()))
        finally:
            s.close()
    (Ex, Hx, ix), (Es, Hs, is_) = out
    assert max_field_rel_l2(Ex, Hx, Es, Hs) < (1e-12 if prec == "fp64" else 1e-5)
    assert len(ix) == len(is_) == 5
    for a, b in zip(ix, is_):
        assert a["step"] == b["step"]
        assert abs(a["E1"] - b["E1"]) <= (1e-12 if prec == "fp64" else 1e-6) * abs(b["E1"])
