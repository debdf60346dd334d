"""Transform schedules: every kernel variant of the y and z passes against the oracle.

The schedule table (mx_set_schedule / mx_schedule) is process-wide per grid shape and
precision, so each test forces the variant on shapes no other test uses and puts the
previous schedules back afterwards.  Tolerances as in test_gpu_parity: FP64 within 1e-12
relative L2 of the oracle, FP32 within 1e-5; the variants run the same line transforms
with a different staging of the tiles, so their results agree far more closely.
"""
import contextlib

import numpy as np
import pytest

import synth
from oracle import scheme
from tests.gpu_util import rel_l2, run_gpu, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
STRIDED = ("y_fwd", "z_fwd", "z_inv", "y_inv")
VARIANTS = [(4, "copy-engine"), (0, "register-prefetch"), (2, "copy-engine-2stage"), (1, "copy-engine-2stage")]


@contextlib.contextmanager
def forced(grid, precision, strided):
    """Force (bps, variant) on the y and z passes of this shape and precision."""
    mx = solver_mod()
    s = mx.Solver(grid.n, grid.lo, grid.hi, 1.0, 1.0, precision, mx.MX_FORM_SPECTRAL)
    try:
        before = s.schedule()
        sched = dict(before)
        for p in STRIDED:
            sched[p] = strided
        s.set_schedule(sched)
        assert all(s.schedule()[p] == tuple(strided) for p in STRIDED)
        yield
    finally:
        s.set_schedule(before)
        s.close()


def _fields(g, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: f"{v[1]}-{v[0]}")
@pytest.mark.parametrize("form", ["literal", "spectral"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_strided_variants_match_oracle(variant, form, prec):
    # y = 64 and z = 48 (lengths that are multiples of 16: every variant applies; the spectral
    # form's load and read run the strided z passes, the literal form the fused one)
    mx = solver_mod()
    g = synth.Grid((20, 64, 48), (0.0, 0.0, 0.0), (TWO_PI, 2.0, 3.0))
    E0, H0 = _fields(g, seed=71)
    eps, mu, h, steps = 1.3, 0.8, 0.037, 3
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_SPECTRAL
    with forced(g, P, variant):
        E, H, _ = run_gpu(g, E0, H0, eps, mu, P, F, h, steps, every=1)
    if form == "literal":
        Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    else:
        Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, h * steps)
    assert rel_l2(E, H, Eo, Ho) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_variants_agree_with_each_other(prec):
    mx = solver_mod()
    g = synth.Grid((12, 32, 80), (0.0, 0.0, 0.0), (TWO_PI, TWO_PI, TWO_PI))
    E0, H0 = _fields(g, seed=72)
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    out = []
    for variant in VARIANTS[:3]:
        with forced(g, P, variant):
            E, H, _ = run_gpu(g, E0, H0, 1.0, 1.0, P, mx.MX_FORM_SPECTRAL, 0.05, 2, every=1)
        out.append((E, H))
    for E, H in out[1:]:
        assert rel_l2(E, H, *out[0]) < (1e-14 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("n", [(16, 512, 8), (10, 512, 6)])  # 8 columns per tile: full / ragged (5 of 8)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_long_lines_default_two_stage(prec, n):
    # lines of 512: the y passes default to the two-stage variant; literal steps against the oracle
    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    g = synth.Grid(n, (0.0, 0.0, 0.0), (1.0, 4.0, 1.0))
    s = mx.Solver(g.n, g.lo, g.hi, 1.0, 1.0, P, mx.MX_FORM_LITERAL)
    try:
        sched = s.schedule()
    finally:
        s.close()
    assert sched["y_fwd"] == (4, "copy-engine-2stage") and sched["y_inv"] == (4, "copy-engine-2stage")
    assert sched["x_r2c"] == (4, "copy-engine") and sched["z_fused"] == (2, "copy-engine")
    E0, H0 = _fields(g, seed=73)
    E, H, _ = run_gpu(g, E0, H0, 2.0, 0.5, P, mx.MX_FORM_LITERAL, 0.02, 3, every=1)
    Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, 2.0, 0.5, 0.02, 3)
    assert rel_l2(E, H, Eo, Ho) < (1e-12 if prec == "fp64" else 1e-5)


def test_set_schedule_rejects_invalid():
    mx = solver_mod()
    g = synth.Grid((8, 16, 16), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    s = mx.Solver(g.n, g.lo, g.hi, 1.0, 1.0, mx.MX_FP32, mx.MX_FORM_SPECTRAL)
    try:
        before = s.schedule()
        bad = [
            {"x_r2c": (4, "copy-engine-2stage")},   # the two-stage variant is for y and z only
            {"z_fused": (3, "copy-engine")},        # fused z: 1 or 2 blocks per SM
            {"y_fwd": (0, "copy-engine")},          # copy-engine variants are persistent
        ]
        for change in bad:
            sched = dict(before)
            sched.update(change)
            with pytest.raises(mx.MaxexpError):
                s.set_schedule(sched)
            assert s.schedule() == before
    finally:
        s.close()
