"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 path within 1e-12 relative L2 of the oracle, invariants
within 1e-12 of the oracle's physical-space values and conserved to
1e-13 (normalised by Cauchy-Schwarz bounds); FP32 path within 1e-5.  On
random fields (every component non-trivial) the L2 bounds hold for each of
the six fields separately.
"""
import numpy as np
import pytest

import synth
from oracle import closed_form as cf
from oracle import invariants as oinv
from oracle import scheme
from tests.gpu_util import inv_diff, inv_scales, max_field_rel_l2, rel_l2, run_gpu, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
# (grid sizes, hi) -- lo = 0.  Covers radix 2/3/5, ragged tiles, the packed
# x column with Mx = 1 and 3, direct (non-commensurate) coefficients, cuboids.
GRIDS = [
    ((16, 16, 16), (TWO_PI, TWO_PI, TWO_PI)),
    ((8, 12, 10), (2.0, 3.0, 2.5)),          # nu^2 ratios 1 : 4/9 : 16/25 -> direct coefficients
    ((2, 4, 6), (1.0, 1.0, 1.0)),            # Mx = 1: only the packed column
    ((6, 20, 12), (TWO_PI, 2 * TWO_PI, TWO_PI)),
    ((20, 10, 24), (3.0, 1.5, 3.0)),
    ((48, 64, 80), (TWO_PI, TWO_PI, TWO_PI)),
]


def _fields(g, seed, divfree):
    if divfree:
        return synth.random_divfree_fields(g, seed=seed, sigma=max(g.n) / 4)
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)


def _mx():
    return solver_mod()


@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("form", ["literal", "spectral"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parity_random_fields(gi, form, prec):
    mx = _mx()
    n, hi = GRIDS[gi]
    g = synth.Grid(n, (0.0, 0.0, 0.0), hi)
    E0, H0 = _fields(g, seed=10 + gi, divfree=False)
    eps, mu, h, steps = 1.7, 0.6, 0.043, 7
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_SPECTRAL
    E, H, inv = run_gpu(g, E0, H0, eps, mu, P, F, h, steps, every=1)
    if form == "literal":
        Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    else:
        Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, h * steps)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert max_field_rel_l2(E, H, Eo, Ho) < tol
    # invariants: first and last record against the oracle's physical-space values
    assert len(inv) == steps + 1
    r0 = oinv.invariants(E0, H0, g.lo, g.hi, eps, mu)
    rn = oinv.invariants(Eo, Ho, g.lo, g.hi, eps, mu)
    sc = inv_scales(r0, eps, mu)
    itol = 1e-12 if prec == "fp64" else 1e-5
    assert inv_diff(inv[0], r0, sc) < itol
    assert inv_diff(inv[-1], rn, sc) < itol
    assert inv[-1]["step"] == steps and abs(inv[-1]["t"] - h * steps) < 1e-15
    for rec in inv:
        assert np.all(rec["E5"] == 0) and np.all(rec["E6"] == 0)
        np.testing.assert_array_equal(rec["M2"], -rec["M1"])


@pytest.mark.parametrize("form", ["literal", "spectral"])
def test_invariants_conserved_fp64(form):
    """Thm 4.1-4.6 on the GPU: every record equal to the first within 1e-13 (normalised)."""
    mx = _mx()
    g = synth.Grid((24, 20, 16), (0, 0, 0), (2.0, 1.7, 1.3))
    E0, H0 = _fields(g, seed=4, divfree=False)
    eps, mu = 2.0, 1.0
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_SPECTRAL
    _, _, inv = run_gpu(g, E0, H0, eps, mu, mx.MX_FP64, F, 0.05, 60, every=1)
    sc = inv_scales(inv[0], eps, mu)
    worst = max(inv_diff(r, inv[0], sc) for r in inv[1:])
    assert worst < 1e-13
    assert inv[0]["divE"] > 0.1  # non-divergence-free input: the conserved value is non-trivial


def test_plane_waves_16cube_100_steps_fp64():
    """16^3 on [0,2pi]^3, eps = mu = 1, 4 plane waves, h = 0.01, 100 steps, invariants every step."""
    mx = _mx()
    g = synth.Grid((16, 16, 16))
    p = synth.plane_wave_params(1, nwaves=4, kmax=3)
    E0, H0 = synth.plane_wave_fields(g, p)
    x, y, z = g.mesh()
    Ee, He = cf.plane_wave_sum(x, y, z, 1.0, p)
    for F in (mx.MX_FORM_LITERAL, mx.MX_FORM_SPECTRAL):
        E, H, inv = run_gpu(g, E0, H0, 1.0, 1.0, mx.MX_FP64, F, 0.01, 100, every=1)
        assert np.abs(E - Ee).max() < 1e-12 and np.abs(H - He).max() < 1e-12
        Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, 1.0, 1.0, 0.01, 100)
        assert rel_l2(E, H, Eo, Ho) < 1e-12
        assert len(inv) == 101
        e1 = cf.plane_wave_energy(p)
        assert max(abs(r["E1"] - e1) for r in inv) < 1e-13 * e1


def test_paper_examples_one_step():
    """Sec. 5.1 and 5.2 with one step of size t_end (the paper's runs), FP64, N = 16."""
    mx = _mx()
    gs = synth.Grid((16, 16, 16), (0, 0, 0), (2, 2, 2))
    Es0, Hs0 = synth.standing_wave_fields(gs)
    gt = synth.Grid((16, 16, 16), (0, 0, 0), (1, 1, 1))
    Et0, Ht0 = synth.travelling_wave_fields(gt)
    for t_end in (1.0, 5.0, 10.0, 15.0, 20.0):
        for F in (mx.MX_FORM_LITERAL, mx.MX_FORM_SPECTRAL):
            E, H, _ = run_gpu(gs, Es0, Hs0, 1.0, 1.0, mx.MX_FP64, F, t_end, 1)
            Ee, He = cf.standing_wave(*gs.mesh(), t_end)
            assert max(np.abs(E - Ee).max(), np.abs(H - He).max()) < 1e-12
            E, H, _ = run_gpu(gt, Et0, Ht0, 1.0, 1.0, mx.MX_FP64, F, t_end, 1)
            Ee, He = cf.travelling_wave(*gt.mesh(), t_end)
            assert max(np.abs(E - Ee).max(), np.abs(H - He).max()) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_buffers_and_roundtrip(prec):
    """Host-pointer load/read; load followed by read returns the input."""
    mx = _mx()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    g = synth.Grid((12, 10, 8), (0, 0, 0), (1.0, 1.0, 1.0))
    E0, H0 = _fields(g, seed=8, divfree=False)
    tol = 1e-14 if prec == "fp64" else 1e-6
    for F in (mx.MX_FORM_LITERAL, mx.MX_FORM_SPECTRAL):
        E, H, inv = run_gpu(g, E0, H0, 1.0, 1.0, P, F, 0.1, 0, device=False)
        assert rel_l2(E, H, E0, H0) < tol
        assert len(inv) == 1
        E, H, inv = run_gpu(g, E0, H0, 1.3, 0.7, P, F, 0.1, 5, device=False)
        Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, 1.3, 0.7, 0.1, 5)
        assert max_field_rel_l2(E, H, Eo, Ho) < (1e-12 if prec == "fp64" else 1e-5)


def test_reversibility_and_zero_step():
    """step(-h, n) after step(h, n) returns the input; h = 0 is the identity."""
    import torch

    mx = _mx()
    g = synth.Grid((32, 16, 24), (0, 0, 0), (TWO_PI, TWO_PI, TWO_PI))
    E0, H0 = _fields(g, seed=9, divfree=True)
    for F in (mx.MX_FORM_LITERAL, mx.MX_FORM_SPECTRAL):
        s = mx.Solver(g.n, g.lo, g.hi, 1.4, 0.9, mx.MX_FP64, F)
        Ed = torch.tensor(E0, device="cuda")
        Hd = torch.tensor(H0, device="cuda")
        s.load(Ed, Hd)
        s.step(0.0, 3, 0)
        s.step(0.37, 25, 5)
        s.step(-0.37, 25, 5)
        s.read(Ed, Hd)
        s.sync()
        t, n = s.time()
        assert n == 53 and abs(t) < 1e-14
        assert rel_l2(Ed.cpu().numpy(), Hd.cpu().numpy(), E0, H0) < 1e-12
        assert len(s.invariants()) == 1 + 10
        s.close()


@pytest.mark.parametrize("n", [128, 160])
def test_fp32_spectral_multichunk_blocks(n):
    """Grids where each block of the pipelined FP32 pass streams many chunks (stage buffers
    reused): FP32 and FP64 spectral forms agree to FP32 round-off."""
    import torch

    mx = _mx()
    res = {}
    for P in (mx.MX_FP64, mx.MX_FP32):
        s = mx.Solver((n, n, n), (0, 0, 0), (TWO_PI,) * 3, 1.3, 0.8, P, mx.MX_FORM_SPECTRAL)
        s.load_random(5, n / 16)
        s.step(0.02, 9, 1)
        dt = torch.float64 if P == mx.MX_FP64 else torch.float32
        E = torch.empty((3, n, n, n), dtype=dt, device="cuda")
        Hh = torch.empty_like(E)
        s.read(E, Hh)
        s.sync()
        res[P] = (E.double().cpu().numpy(), Hh.double().cpu().numpy(), s.invariants())
        s.close()
    E64, H64, i64 = res[mx.MX_FP64]
    E32, H32, i32 = res[mx.MX_FP32]
    assert max_field_rel_l2(E32, H32, E64, H64) < 1e-6
    sc = inv_scales(i64[0], 1.3, 0.8)
    assert max(inv_diff(a, b, sc) for a, b in zip(i32, i64)) < 1e-6


def test_deterministic_invariants():
    """Same input, same launch: bitwise identical invariant records and fields."""
    mx = _mx()
    g = synth.Grid((32, 32, 32))
    E0, H0 = _fields(g, seed=12, divfree=True)
    runs = [run_gpu(g, E0, H0, 1.0, 1.0, mx.MX_FP32, mx.MX_FORM_SPECTRAL, 0.02, 10) for _ in range(2)]
    for a, b in zip(runs[0][2], runs[1][2]):
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(runs[0][0], runs[1][0])


def test_errors_are_status_codes():
    mx = _mx()
    import ctypes as C

    h = C.c_void_p()
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    s = mx.Solver((8, 8, 8), (0, 0, 0), (1, 1, 1), 1.0, 1.0)
    assert mx.mx_step(s.handle, 0.1, 1, 1) == mx.MX_E_STATE  # before load
    buf = np.zeros((3, 8, 8, 8))
    s.load(buf, buf)
    assert mx.mx_step(s.handle, float("nan"), 1, 1) == mx.MX_E_INVAL
    assert mx.mx_step(s.handle, 0.1, -1, 1) == mx.MX_E_INVAL
    s.close()
    assert mx.mx_create(C.byref(h), 14, 8, 8, lo, hi, 1.0, 1.0, 0, 0, None) == mx.MX_E_UNSUPPORTED_N
    assert not h.value


def _omega(Ea, Ha, Eb, Hb, eps, mu):
    """Symplectic form of Thm 4.5 in u = sqrt(mu) H, v = sqrt(eps) E: <v_a, u_b> - <u_a, v_b>."""
    return float(np.sum(np.sqrt(eps) * Ea * np.sqrt(mu) * Hb) - np.sum(np.sqrt(mu) * Ha * np.sqrt(eps) * Eb))


@pytest.mark.parametrize("form", ["literal", "spectral"])
def test_symplectic_form_preserved_fp64(form):
    """Thm 4.5 on the GPU: the step preserves dE ^ dH, omega(R a, R b) = omega(a, b), for two
    independent states (not divergence free, every wavenumber populated)."""
    mx = _mx()
    g = synth.Grid((12, 10, 8), (0, 0, 0), (1.0, 1.4, 0.9))
    rng = np.random.default_rng(45)
    Ea, Ha, Eb, Hb = (rng.standard_normal((3,) + g.shape) for _ in range(4))
    eps, mu = 1.6, 0.7
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_SPECTRAL
    Ea1, Ha1, _ = run_gpu(g, Ea, Ha, eps, mu, mx.MX_FP64, F, 0.3, 10, every=0)
    Eb1, Hb1, _ = run_gpu(g, Eb, Hb, eps, mu, mx.MX_FP64, F, 0.3, 10, every=0)
    w0 = _omega(Ea, Ha, Eb, Hb, eps, mu)
    w1 = _omega(Ea1, Ha1, Eb1, Hb1, eps, mu)
    na = np.sqrt(eps * np.sum(Ea ** 2) + mu * np.sum(Ha ** 2))
    nb = np.sqrt(eps * np.sum(Eb ** 2) + mu * np.sum(Hb ** 2))
    assert abs(w0) > 1e-3 * na * nb  # not trivially zero
    assert abs(w1 - w0) < 1e-12 * na * nb


# the longest lines of each radix family in every direction: x rows of 512 and 320 reals,
# y and z lines of 384 (fused z plan of 3 * 2^a) and 320 (z without a fused plan)
EDGE_GRIDS = [(512, 6, 8), (320, 4, 6), (8, 384, 6), (6, 8, 384), (8, 320, 10), (10, 6, 320)]


@pytest.mark.parametrize("n", EDGE_GRIDS)
@pytest.mark.parametrize("form", ["literal", "spectral"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parity_longest_lines(n, form, prec):
    mx = _mx()
    g = synth.Grid(n, (0.0, 0.0, 0.0), (2.0, 3.0, 2.5))
    E0, H0 = _fields(g, seed=sum(n), divfree=False)
    eps, mu, h, steps = 1.3, 0.8, 0.021, 4
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_SPECTRAL
    E, H, inv = run_gpu(g, E0, H0, eps, mu, P, F, h, steps, every=1)
    if form == "literal":
        Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    else:
        Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, h * steps)
    assert max_field_rel_l2(E, H, Eo, Ho) < (1e-12 if prec == "fp64" else 1e-5)
    assert len(inv) == steps + 1


def test_spectral_convergence_thm34_gpu():
    """Thm 3.4 on the GPU (literal FP64, 10 steps): for smooth, non-band-limited data the error
    against a 48^3 run decays faster than any power of N; the 48^3 reference is the GPU's too,
    and every grid also matches the oracle."""
    mx = _mx()

    def fields(n):
        g = synth.Grid((n, n, n))
        x, y, z = g.mesh()
        a = np.exp(np.sin(x)) * np.exp(np.cos(y))  # A = (0, 0, a cos z); E = curl A, H = 0
        E = np.stack([a * (-np.sin(y)) * np.cos(z), -(a * np.cos(x)) * np.cos(z), 0 * x])
        return g, E, 0 * E

    h, steps = 0.07, 10
    gF, EF, HF = fields(48)
    EfT, HfT, _ = run_gpu(gF, EF, HF, 1.0, 1.0, mx.MX_FP64, mx.MX_FORM_LITERAL, h, steps, every=0)
    errs = []
    for n in (8, 12, 16, 24):
        g, E, H = fields(n)
        Et, Ht, _ = run_gpu(g, E, H, 1.0, 1.0, mx.MX_FP64, mx.MX_FORM_LITERAL, h, steps, every=0)
        Eo, Ho = scheme.step(E, H, g.lo, g.hi, 1.0, 1.0, h, steps)
        assert rel_l2(Et, Ht, Eo, Ho) < 1e-12
        s = 48 // n
        errs.append(np.sqrt(np.mean((Et - EfT[:, ::s, ::s, ::s]) ** 2) + np.mean((Ht - HfT[:, ::s, ::s, ::s]) ** 2)))
    assert errs[-1] < 1e-6 * errs[0]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(n2 / n1) for i, (n1, n2) in enumerate([(8, 12), (12, 16), (16, 24)])]
    assert rates[-1] > rates[0] > 2.0
